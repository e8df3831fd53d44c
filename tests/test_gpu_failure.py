"""Failure path of the handles, driven from the host: lee_test_inject_cuda_error makes one checked
CUDA call report an error although it succeeded, so no GPU fault is involved.  After the reported
error the handle is poisoned: the failing call returns LEE_ERR_CUDA, every later call on that
handle LEE_ERR_POISONED, destroy still succeeds, and a new handle works normally."""
import numpy as np
import pytest

from paper_1601_08103_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.fixture
def inject(gpu_lib):
    yield gpu_lib.lee_test_inject_cuda_error
    gpu_lib.lee_test_inject_cuda_error(-1)


def _expect(lee, status, fn, *args):
    with pytest.raises(lee.LeeError) as e:
        fn(*args)
    assert e.value.status == status, (fn, e.value)
    return e.value


@pytest.mark.parametrize("after", [0, 1, 2])
def test_injected_error_poisons_the_solver(gpu_lib, inject, after):
    lee = gpu_lib
    shape = (64, 32, 1)
    cells = shape[0] * shape[1]
    rho, u, th = inputs.random_fields(shape, 2, 3)
    sv = lee.Solver("D2Q5", shape, 0.6, storage="f32")
    try:
        sv.init_fields(rho, u, th)
        sv.step(2)
        inject(after)
        err = _expect(lee, lee.LEE_ERR_CUDA, sv.step, 9)
        assert "unknown" in str(err).lower() or lee.lee_lbm_last_error(sv.h)
        inject(-1)
        mr, out, g = np.empty(cells), np.empty(6), np.empty((5, cells))
        for fn, args in ((sv.step, (1,)), (sv.moments, (mr,)), (sv.reduce, (out,)), (sv.get_populations, (g,)),
                         (sv.set_populations, (g,)), (sv.init_fields, (rho, u, th)), (sv.sync, ())):
            _expect(lee, lee.LEE_ERR_POISONED, fn, *args)
    finally:
        sv.close()  # destroy succeeds on a poisoned handle
    # the process and the device are fine: a new handle runs
    with lee.Solver("D2Q5", shape, 0.6, storage="f32") as ok:
        ok.init_fields(rho, u, th)
        ok.step(5)
        red = np.empty(6)
        ok.reduce(red)
    assert np.isfinite(red).all() and red[-1] == 0


def test_injected_error_poisons_the_batch(gpu_lib, inject):
    lee = gpu_lib
    doms = [(64, 64, 0.6), (128, 64, 0.8)]
    b = lee.Batch("D2Q5", "f32", doms)
    try:
        for d, (nx, ny, _) in enumerate(doms):
            b.init_fields(d, *inputs.random_fields((nx, ny, 1), 2, d))
        b.step(2)
        inject(1)
        _expect(lee, lee.LEE_ERR_CUDA, b.step, 8)
        inject(-1)
        r = np.empty(64 * 64)
        for fn, args in ((b.step, (1,)), (b.moments, (0, r)), (b.reduce, (0, np.empty(6))), (b.sync, ())):
            _expect(lee, lee.LEE_ERR_POISONED, fn, *args)
    finally:
        b.close()


def test_injected_error_poisons_the_network(gpu_lib, inject):
    import torch

    from oracle import mlp as omlp

    lee = gpu_lib
    m = lee.Mlp(omlp.init_params(1).astype(np.float32))
    try:
        x = torch.zeros((64, lee.MLP_IN), dtype=torch.float32, device="cuda")
        y = torch.zeros(64, dtype=torch.float32, device="cuda")
        m.forward(x, 64, y)
        inject(0)
        _expect(lee, lee.LEE_ERR_CUDA, m.forward, x, 64, y)
        inject(-1)
        _expect(lee, lee.LEE_ERR_POISONED, m.forward, x, 64, y)
        _expect(lee, lee.LEE_ERR_POISONED, m.loss_grad, x, y, 64)
        _expect(lee, lee.LEE_ERR_POISONED, m.adam_step, 1e-3)
    finally:
        m.close()
