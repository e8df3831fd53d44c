"""Slab decomposition on the GPU (LEE_BC_SLAB, include/lee_lbm.h), through the C ABI.

A periodic domain cut along its last axis into 1-4 slabs of uneven thickness, all held in this
process on one GPU: lee_lbm_slab_step packs the crossing populations of every slab, copies each
message into its receiver's own halo buffer and unpacks it, then steps every slab.  The assembled
state equals the single-domain run of the same storage bit for bit (the per-cell arithmetic is the
same), and FP64 is within 1e-12 of the oracle.  The Python ring (SlabRing over GpuSlab) gives the
same bits with a transport that copies between two slabs' torch views."""
import numpy as np
import pytest

import oracle
from paper_1601_08103_gb300 import inputs, slab

from test_gpu_parity import perm_to_lib, rel_l2

pytestmark = pytest.mark.gpu


def _slab_shape(shape, D, count):
    s = list(shape)
    s[D - 1] = count
    return tuple(s)


def _cut_fields(fields, shape, D, start, count):
    """The slab's part of FP64 fields rho[cells], u[D][cells], theta[cells]."""
    nx, ny, nz = shape
    dims = (nz, ny, nx) if D == 3 else (ny, nx)
    rho, u, th = fields
    take = lambda a: np.ascontiguousarray(a.reshape(dims)[start:start + count]).ravel()
    return take(rho), np.stack([take(u[a]) for a in range(D)]), take(th)


def _assemble(solvers, q, shape, D):
    parts = []
    for sv in solvers:
        g = np.empty((q, sv.cells))
        sv.get_populations(g)
        nx, ny, nz = sv.shape
        parts.append(g.reshape((q, nz, ny, nx) if D == 3 else (q, ny, nx)))
    return np.concatenate(parts, axis=1).reshape(q, -1)


CASES = [("D2Q5", (256, 64, 1), 0.6, 9), ("D2Q5_DI", (132, 30, 1), 0.52, 6), ("D3Q7", (64, 32, 40), 0.55, 7),
         ("D3Q19", (32, 16, 20), 0.7, 5), ("D3Q13", (24, 10, 11), 0.8, 4)]


@pytest.mark.parametrize("name,shape,tau,n", CASES)
@pytest.mark.parametrize("storage", ["f64", "f32", "f16"])
@pytest.mark.parametrize("count", [1, 2, 3, 4])
def test_slabs_equal_the_single_domain(gpu_lib, monkeypatch, name, shape, tau, n, storage, count):
    lee = gpu_lib
    # one step per launch for the single-domain run too: 16-bit storage otherwise fuses four steps
    # per launch on periodic 2D grids and rounds once per launch (FP32 fusion gives the same bits)
    monkeypatch.setenv("LEE_TB_STEPS", "1")
    info = lee.lee_velset_info(name)
    D, q = info["D"], info["q"]
    cells = int(np.prod(shape))
    fields = inputs.random_fields(shape, D, 90 + count)
    with lee.Solver(name, shape, tau, storage=storage, store_scale=1024.0) as sv:
        sv.init_fields(*fields)
        sv.step(n)
        want = np.empty((q, cells))
        sv.get_populations(want)
    slabs = []
    try:
        for start, planes in slab.partition(shape[D - 1], count):
            sv = lee.Solver(name, _slab_shape(shape, D, planes), tau, storage=storage, bc="slab", store_scale=1024.0)
            slabs.append(sv)
            sv.init_fields(*_cut_fields(fields, shape, D, start, planes))
        lee.lee_lbm_slab_step(slabs, n)
        got = _assemble(slabs, q, shape, D)
        crossing, plane, nbytes = slabs[0].slab_info()
        assert crossing == sum(1 for c in info["c"] if c[D - 1] == 1)
        assert plane == (shape[0] * shape[1] if D == 3 else shape[0])
    finally:
        for sv in slabs:
            sv.close()
    assert np.array_equal(got, want), (name, storage, count)
    if storage == "f64":
        g = oracle.step(name, shape, tau, oracle.equilibrium(name, *fields), n)
        ref = oracle.post_state(name, shape, tau, g)[perm_to_lib(lee, name)]
        assert rel_l2(got, ref) <= 1e-12


def test_python_ring_on_gpu_slabs(gpu_lib):
    """The ring of paper_1601_08103_gb300.slab with GpuSlab views of the library's halo buffers:
    a one-rank DistTransport (gloo group of one process) for a single slab, and a two-slab
    exchange written out with the same buffers; both equal the single-domain run."""
    import os

    import torch
    import torch.distributed as dist

    lee = gpu_lib
    name, shape, tau, n = "D3Q7", (64, 16, 24), 0.6, 6
    fields = inputs.random_fields(shape, 3, 5)
    stream = torch.cuda.current_stream()
    with lee.Solver(name, shape, tau, storage="f32") as sv:
        sv.init_fields(*fields)
        sv.step(n)
        want = np.empty((7, int(np.prod(shape))))
        sv.get_populations(want)
    # one slab, one-rank group: the transport copies its own messages across
    import socket

    sk = socket.socket()
    sk.bind(("127.0.0.1", 0))
    port = sk.getsockname()[1]
    sk.close()
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=0, world_size=1)
    try:
        with lee.Solver(name, shape, tau, storage="f32", bc="slab", stream=stream) as one:
            one.init_fields(*fields)
            slab.SlabRing(slab.GpuSlab(one), slab.DistTransport()).step(n)
            got = np.empty_like(want)
            one.get_populations(got)
        assert np.array_equal(got, want)
    finally:
        dist.destroy_process_group()
    # two slabs: pack both, swap the messages through the torch views, unpack, step
    (s0, c0), (s1, c1) = slab.partition(shape[2], 2)
    a = lee.Solver(name, (64, 16, c0), tau, storage="f32", bc="slab", stream=stream)
    b = lee.Solver(name, (64, 16, c1), tau, storage="f32", bc="slab", stream=stream)
    try:
        a.init_fields(*_cut_fields(fields, shape, 3, s0, c0))
        b.init_fields(*_cut_fields(fields, shape, 3, s1, c1))
        ga, gb = slab.GpuSlab(a), slab.GpuSlab(b)
        for _ in range(n):
            ga.pack()
            gb.pack()
            (a_lo, a_hi, a_rlo, a_rhi), (b_lo, b_hi, b_rlo, b_rhi) = ga.buffers(), gb.buffers()
            b_rhi.copy_(a_lo)  # a's lower neighbour is b (periodic), its upper neighbour too
            b_rlo.copy_(a_hi)
            a_rhi.copy_(b_lo)
            a_rlo.copy_(b_hi)
            ga.unpack()
            gb.unpack()
            ga.step1()
            gb.step1()
        got2 = _assemble([a, b], 7, shape, 3)
    finally:
        a.close()
        b.close()
    assert np.array_equal(got2, want)


def test_slab_handles_reject_misuse(gpu_lib):
    lee = gpu_lib
    with lee.Solver("D2Q5", (64, 8, 1), 0.6, storage="f32", bc="slab") as a, \
            lee.Solver("D2Q5", (64, 8, 1), 0.7, storage="f32", bc="slab") as b, \
            lee.Solver("D2Q5", (64, 8, 1), 0.6, storage="f32") as c:
        with pytest.raises(lee.LeeError) as e:
            a.step(2)  # every step needs a fresh exchange
        assert e.value.status == lee.LEE_ERR_INVALID_ARGUMENT
        for group in ([a, b], [a, c], [a, a]):  # other tau; not a slab; listed twice
            with pytest.raises(lee.LeeError):
                lee.lee_lbm_slab_step(group, 1)
        with pytest.raises(lee.LeeError):
            c.slab_pack()
