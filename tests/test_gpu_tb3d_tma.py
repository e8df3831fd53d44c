"""The TMA-fed 3D two-step tile (paper_1601_08103_gb300/csrc/tb3d_tma.cuh) on the GPU, through the
C ABI.

- FP32: a launch equals two single steps bit for bit (LEE_SINGLE_STEP=1 reference), and equals
  the register-fed tile (LEE_T3_TMA=0) bit for bit.
- BFP16: equals the register-fed two-step tile bit for bit (both decode, take two FP32 steps and
  encode); the one-launch decomposition itself is checked in test_gpu_bfp16.py.
- Shapes cover one to three 128-column strips, first and last tile rows (rows wrapping around y
  through the single-row boxes), several tile rows, z segments and nz of 1 and 2 (planes wrapping
  onto themselves), both the graph-captured and the direct launches.
- The solver takes it only when LEE_T3_TMA=1 asks for it (it measured slower than the register-fed
  tile); grids it cannot take keep their kernels.
- Its bounded stage wait: lee_test_inject_stage_timeout makes the first stage of every launch
  short of 16 announced bytes; the wait runs out (20 ms), the handle reports LEE_ERR_TIMEOUT and
  is poisoned, destroy succeeds and a new handle runs normally.  No GPU fault or hang is involved.
"""
import numpy as np
import pytest

import oracle
from paper_1601_08103_gb300 import inputs

from test_gpu_parity import rel_l2

pytestmark = pytest.mark.gpu

SHAPES = [(128, 16, 6), (256, 24, 9), (384, 16, 3), (128, 32, 1), (128, 16, 2), (128, 48, 20)]


def _run(lee, monkeypatch, env, name, shape, tau, storage, n, fields):
    for k in ("LEE_T3_TMA", "LEE_TB_STEPS", "LEE_SINGLE_STEP"):
        monkeypatch.delenv(k, raising=False)
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    q = lee.lee_velset_info(name)["q"]
    with lee.Solver(name, shape, tau, storage=storage) as sv:
        spl = sv.steps_per_launch
        sv.init_fields(*fields)
        sv.step(n)
        g = np.empty((q, int(np.prod(shape))))
        sv.get_populations(g)
    return g, spl


@pytest.mark.parametrize("name", ["D3Q7", "D3Q7_DI"])
@pytest.mark.parametrize("shape", SHAPES)
def test_fp32_tma_tile_equals_single_steps(gpu_lib, monkeypatch, name, shape):
    lee = gpu_lib
    fields = inputs.random_fields(shape, 3, 17)
    n = 10  # eight steps in a captured graph, then one direct launch
    g_t, spl = _run(lee, monkeypatch, {"LEE_T3_TMA": "1"}, name, shape, 0.57, "f32", n, fields)
    assert spl == 2
    g_1, spl1 = _run(lee, monkeypatch, {"LEE_SINGLE_STEP": "1"}, name, shape, 0.57, "f32", n, fields)
    assert spl1 == 1
    g_r, _ = _run(lee, monkeypatch, {"LEE_T3_TMA": "0"}, name, shape, 0.57, "f32", n, fields)
    assert np.array_equal(g_t, g_1)
    assert np.array_equal(g_t, g_r)


@pytest.mark.parametrize("name", ["D3Q7", "D3Q7_DI"])
@pytest.mark.parametrize("shape", SHAPES)
def test_bfp16_tma_tile_equals_register_tile(gpu_lib, monkeypatch, name, shape):
    lee = gpu_lib
    fields = inputs.random_fields(shape, 3, 23)
    n = 10
    g_t, spl = _run(lee, monkeypatch, {"LEE_T3_TMA": "1"}, name, shape, 0.55, "bfp16", n, fields)
    assert spl == 2
    g_r, spl_r = _run(lee, monkeypatch, {"LEE_T3_TMA": "0", "LEE_TB_STEPS": "2"}, name, shape, 0.55, "bfp16", n,
                      fields)
    assert spl_r == 2
    assert np.array_equal(g_t, g_r)


def test_kernel_choice(gpu_lib, monkeypatch):
    lee = gpu_lib
    for k in ("LEE_T3_TMA", "LEE_TB_STEPS", "LEE_SINGLE_STEP"):
        monkeypatch.delenv(k, raising=False)
    # BFP16 runs one step per launch by default; LEE_T3_TMA=1 gives the TMA-fed two-step tile where
    # the grid allows it
    for shape in ((384, 384, 384), (128, 16, 4)):
        with lee.Solver("D3Q7", shape, 0.6, storage="bfp16") as sv:
            assert sv.steps_per_launch == 1, shape
    monkeypatch.setenv("LEE_T3_TMA", "1")
    for shape, want in (((384, 384, 384), 2), ((128, 16, 4), 2), ((136, 16, 4), 1), ((128, 12, 4), 1),
                        ((128, 8, 4), 1)):
        with lee.Solver("D3Q7", shape, 0.6, storage="bfp16") as sv:
            assert sv.steps_per_launch == want, shape
    # FP32 keeps two steps per launch either way; D3Q19 has no two-step tile
    with lee.Solver("D3Q7", (128, 16, 4), 0.6, storage="f32") as sv:
        assert sv.steps_per_launch == 2
    with lee.Solver("D3Q19", (128, 16, 4), 0.6, storage="bfp16") as sv:
        assert sv.steps_per_launch == 1


@pytest.mark.parametrize("name", ["D3Q7", "D3Q7_DI"])
def test_bfp16_tma_tile_against_oracle(gpu_lib, monkeypatch, name):
    """Smooth pulse, 40 steps: within the storage bound of one rounding per two steps."""
    lee = gpu_lib
    for k in ("LEE_TB_STEPS", "LEE_SINGLE_STEP"):
        monkeypatch.delenv(k, raising=False)
    monkeypatch.setenv("LEE_T3_TMA", "1")
    shape, tau, n = (128, 32, 24), 0.55, 40
    rho = inputs.gaussian_pulse(shape, 1e-3, 4.0, [60.0, 14.0, 11.0])
    u, th = inputs.zero_rest(3, int(np.prod(shape)))
    with lee.Solver(name, shape, tau, storage="bfp16") as sv:
        assert sv.steps_per_launch == 2
        sv.init_fields(rho, u, th)
        sv.step(n)
        m = np.empty(int(np.prod(shape)))
        sv.moments(m)
    g = oracle.step(name, shape, tau, oracle.equilibrium(name, rho, u, th), n)
    want = oracle.moments(name, g)[0]
    err = rel_l2(m, want)
    assert 0 < err <= 4 * 2.0 ** -15 * np.sqrt(10 * n / 2), err


@pytest.mark.parametrize("storage", ["bfp16", "f32"])
def test_stage_timeout_poisons_the_handle(gpu_lib, monkeypatch, storage):
    lee = gpu_lib
    monkeypatch.setenv("LEE_T3_TMA", "1")
    monkeypatch.delenv("LEE_TB_STEPS", raising=False)
    monkeypatch.delenv("LEE_SINGLE_STEP", raising=False)
    shape = (128, 16, 4)
    cells = int(np.prod(shape))
    fields = inputs.random_fields(shape, 3, 5)
    sv = lee.Solver("D3Q7", shape, 0.6, storage=storage)
    try:
        assert sv.steps_per_launch == 2
        sv.init_fields(*fields)
        sv.step(2)
        sv.sync()
        lee.lee_test_inject_stage_timeout(True, 20_000_000)
        try:
            sv.step(2)  # one direct launch whose first stage never completes
        finally:
            lee.lee_test_inject_stage_timeout(False)
        with pytest.raises(lee.LeeError) as e:
            sv.sync()
        assert e.value.status == lee.LEE_ERR_TIMEOUT
        g = np.empty((7, cells))
        for fn, args in ((sv.step, (2,)), (sv.get_populations, (g,)), (sv.sync, ())):
            with pytest.raises(lee.LeeError) as e:
                fn(*args)
            assert e.value.status == lee.LEE_ERR_POISONED
    finally:
        sv.close()
    # the context is fine: a new handle on the same tile gives the single-step result
    with lee.Solver("D3Q7", shape, 0.6, storage="f32") as a:
        a.init_fields(*fields)
        a.step(6)
        ga = np.empty((7, cells))
        a.get_populations(ga)
    monkeypatch.setenv("LEE_SINGLE_STEP", "1")
    with lee.Solver("D3Q7", shape, 0.6, storage="f32") as b:
        b.init_fields(*fields)
        b.step(6)
        gb = np.empty((7, cells))
        b.get_populations(gb)
    assert np.array_equal(ga, gb)


def test_stage_timeout_hook_rejects_bad_arguments(gpu_lib):
    lee = gpu_lib
    for on, ns in ((2, 0), (-1, 0), (1, -5), (1, 10**11)):
        assert lee.load().lee_test_inject_stage_timeout(on, ns) == lee.LEE_ERR_INVALID_ARGUMENT
