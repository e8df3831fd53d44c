"""BFP16 storage (block floating point, include/lee_lbm.h) on the GPU, through the C ABI.

- What the library stores equals the format reference (oracle/bfp.py) bit for bit.
- Every kernel that writes BFP16 state -- the one-step kernel (vector and scalar paths, periodic,
  zero-incoming and sponge edges), the 2D K-level tiles and the 3D two-step tile -- computes one
  launch of k steps as: decode the state, k FP32 steps, encode.  Checked bit for bit against the
  library's own FP32 path (bit-identical to single FP32 steps) and import encoding.
- Against the FP64 oracle the error stays within the storage bound and at least four times below
  FP16's on the same smooth-pulse runs.
"""
import numpy as np
import pytest

import oracle
from oracle import bfp
from paper_1601_08103_gb300 import inputs

from test_gpu_parity import assert_close, perm_to_lib, rel_l2, run_pair

pytestmark = pytest.mark.gpu

SETS = ["D1Q3", "D2Q5", "D2Q5_DI", "D3Q7", "D3Q9", "D3Q13", "D3Q19", "D3Q7_DI"]


def _shape(D, ragged=False):
    if D == 1:
        return (1027, 1, 1) if ragged else (1024, 1, 1)
    if D == 2:
        return (129, 33, 1) if ragged else (256, 40, 1)
    return (13, 11, 9) if ragged else (40, 10, 7)


@pytest.mark.parametrize("name", SETS)
@pytest.mark.parametrize("ragged", [False, True])
def test_stored_values_follow_the_format(gpu_lib, name, ragged):
    lee = gpu_lib
    info = lee.lee_velset_info(name)
    shape = _shape(info["D"], ragged)
    cells = int(np.prod(shape))
    rng = np.random.default_rng(11)
    # populations of very different magnitudes per region, a zero stretch and a far-field tail
    g = rng.normal(size=(info["q"], cells)) * 10.0 ** rng.uniform(-9, -2, size=(1, cells))
    g[:, cells // 3: cells // 3 + 40] = 0.0
    with lee.Solver(name, shape, 0.6, storage="bfp16") as sv:
        sv.set_populations(g)
        got = np.empty_like(g)
        sv.get_populations(got)
    pad = (-cells) % 8  # cells past the grid in the last block are encoded as zeros
    v32 = np.concatenate([g.astype(np.float32), np.zeros((info["q"], pad), np.float32)], axis=1)
    want = bfp.round_trip(v32)[:, :cells]
    assert np.array_equal(got, want)


# (set, shape, bc, steps per launch)
CASES = [("D2Q5", (256, 40, 1), "periodic", 1), ("D2Q5", (256, 40, 1), "periodic", 4),
         ("D2Q5", (264, 37, 1), "periodic", 4), ("D2Q5_DI", (384, 130, 1), "periodic", 3),
         ("D2Q5", (16, 5, 1), "periodic", 4), ("D2Q5", (260, 37, 1), "periodic", 1),
         ("D3Q7", (128, 10, 5), "periodic", 2), ("D3Q7_DI", (136, 9, 6), "periodic", 2),
         ("D3Q7", (128, 8, 40), "periodic", 2), ("D3Q7", (40, 10, 7), "periodic", 1),
         ("D3Q19", (64, 6, 5), "periodic", 1), ("D3Q13", (13, 11, 9), "periodic", 1),
         ("D1Q3", (1024, 1, 1), "periodic", 1), ("D1Q3", (1000, 1, 1), "open_sponge", 1),
         ("D2Q5", (64, 48, 1), "open_zero", 1), ("D2Q5", (64, 48, 1), "open_sponge", 1),
         ("D3Q19", (40, 10, 9), "open_sponge", 1), ("D3Q7", (13, 11, 9), "periodic", 1),
         ("D3Q19", (13, 11, 9), "periodic", 1), ("D3Q13", (16, 11, 9), "periodic", 1),
         ("D2Q5", (13, 40, 1), "periodic", 1), ("D3Q9", (13, 11, 9), "periodic", 1)]


@pytest.mark.parametrize("name,shape,bc,k", CASES)
def test_one_launch_is_decode_fp32_steps_encode(gpu_lib, monkeypatch, name, shape, bc, k):
    lee = gpu_lib
    info = lee.lee_velset_info(name)
    cells = int(np.prod(shape))
    kw = dict(sponge_width=3, sponge_strength=0.5) if bc == "open_sponge" else {}
    monkeypatch.setenv("LEE_TB_STEPS", str(k) if k > 1 else "1")
    rho, u, th = inputs.random_fields(shape, info["D"], 41)
    with lee.Solver(name, shape, 0.55, storage="bfp16", bc=bc, **kw) as a:
        assert a.steps_per_launch == k
        a.init_fields(rho, u, th)
        a.step(2 * k + (1 if k == 1 else 0))  # a state a few steps in
        g0 = np.empty((info["q"], cells))
        a.get_populations(g0)
        a.step(k)  # exactly one launch
        g1 = np.empty_like(g0)
        a.get_populations(g1)
    with lee.Solver(name, shape, 0.55, storage="f32", bc=bc, **kw) as b:
        b.set_populations(g0)  # the decoded values are FP32 values: stored exactly
        b.step(k)
        gb = np.empty_like(g0)
        b.get_populations(gb)
    with lee.Solver(name, shape, 0.55, storage="bfp16", bc=bc, **kw) as c:
        c.set_populations(gb)  # the library's encoding of the FP32 result
        gc = np.empty_like(g0)
        c.get_populations(gc)
    if not np.array_equal(g1, gc):
        pad = (-cells) % 8
        ref = bfp.round_trip(np.concatenate([gb.astype(np.float32), np.zeros((info["q"], pad), np.float32)], 1))
        ref = ref[:, :cells]
        bad = np.argwhere(g1 != gc)
        lines = [f"{len(bad)} differ; stored == format(FP32 step): {np.array_equal(g1, ref)}; "
                 f"import == format: {np.array_equal(gc, ref)}"]
        for i, x in bad[:12]:
            lines.append(f"  v{i} cell {x} (x {x % shape[0]}, row {x // shape[0]}): kernel {g1[i, x]!r} "
                         f"import {gc[i, x]!r} fp32 {gb[i, x]!r} block {x // 8}")
        raise AssertionError("\n".join(lines))


def test_default_launch_shapes(gpu_lib, monkeypatch):
    lee = gpu_lib
    monkeypatch.delenv("LEE_TB_STEPS", raising=False)
    monkeypatch.delenv("LEE_SINGLE_STEP", raising=False)
    for name, shape, want in (("D2Q5", (2048, 2048, 1), 4), ("D2Q5", (260, 64, 1), 1), ("D3Q7", (384, 384, 384), 1),
                              ("D3Q7", (132, 8, 8), 1), ("D3Q19", (64, 64, 64), 1), ("D1Q3", (1024, 1, 1), 1)):
        with lee.Solver(name, shape, 0.6, storage="bfp16") as sv:
            assert sv.steps_per_launch == want, (name, shape)
    with pytest.raises(lee.LeeError) as e:
        lee.Solver("D2Q5", (64, 64, 1), 0.6, storage="bfp16", bc="open_learned")
    assert e.value.status == lee.LEE_ERR_UNSUPPORTED


@pytest.mark.parametrize("name", ["D1Q3", "D2Q5", "D2Q5_DI", "D3Q7", "D3Q19", "D3Q7_DI"])
@pytest.mark.parametrize("bc", ["periodic", "open_sponge"])
def test_error_against_oracle_beats_fp16(gpu_lib, name, bc):
    """Smooth pulse (the workload of the 16-bit configuration), 40 steps at tau = 0.55: BFP16
    against the FP64 oracle within its storage bound, and at least four times below FP16."""
    lee = gpu_lib
    s = oracle.velset(name)
    shape = _shape(s.D)
    if bc == "open_sponge" and s.D == 3:
        shape = (40, 10, 9)
    cells = int(np.prod(shape))
    rho = inputs.gaussian_pulse(shape, 1e-3, 3.0, [n / 2.3 for n in shape])
    u, th = inputs.zero_rest(s.D, cells)
    n = 40
    kw = dict(sponge_w=3, smax=0.4) if bc == "open_sponge" else {}
    errs = {}
    for storage in ("bfp16", "f16"):
        r = run_pair(lee, name, shape, 0.55, n, storage=storage, bc=bc, fields=(rho, u, th), **kw)
        errs[storage] = rel_l2(r["m_gpu"][0], r["m_ora"][0])
    bound = 4 * 2.0 ** -15 * np.sqrt(10 * n)
    assert 0 < errs["bfp16"] <= bound, errs
    assert errs["bfp16"] * 4 <= errs["f16"], errs


@pytest.mark.parametrize("name", ["D2Q5", "D3Q7", "D3Q19"])
def test_reduction_of_bfp16_state(gpu_lib, name):
    """The FP64 reduction decodes the stored values: it equals the oracle's sums of the decoded
    populations; conservation holds to the storage error."""
    lee = gpu_lib
    s = oracle.velset(name)
    shape = _shape(s.D)
    cells = int(np.prod(shape))
    p = perm_to_lib(lee, name)
    rho, u, th = inputs.random_fields(shape, s.D, 5)
    with lee.Solver(name, shape, 0.6, storage="bfp16") as sv:
        sv.init_fields(rho, u, th)
        r0 = np.empty(s.D + 4)
        sv.reduce(r0)
        sv.step(12)
        g = np.empty((s.q, cells))
        sv.get_populations(g)
        red = np.empty(s.D + 4)
        sv.reduce(red)
    want = oracle.reduce(name, g[np.argsort(p)])
    np.testing.assert_allclose(red[:-1], want[:-1], rtol=1e-12, atol=1e-15 * np.abs(g).sum())
    assert red[-1] == 0
    # sum rho', momentum and energy: conserved up to the rounding of the stored values (at most
    # 2^-15 of a block maximum per value and store, summed like a random walk over 13 stores)
    walk = 4 * 2.0 ** -15 * np.abs(g).max() * np.sqrt(13 * cells * s.q)
    np.testing.assert_allclose(red[: s.D + 2], r0[: s.D + 2], atol=walk)


def test_nonfinite_block_is_counted(gpu_lib):
    lee = gpu_lib
    name, shape = "D2Q5", (256, 40, 1)
    cells = int(np.prod(shape))
    g = inputs.random_populations(5, cells, seed=3)
    g[2, 100] = np.nan
    g[4, cells - 1] = np.inf
    with lee.Solver(name, shape, 0.6, storage="bfp16") as sv:
        sv.set_populations(g)
        stored = np.empty_like(g)
        sv.get_populations(stored)
        red = np.empty(6)
        sv.reduce(red)
        assert not sv.check_finite()
    # the whole 8-cell block of each bad value decodes as NaN
    assert np.isnan(stored[2, 96:104]).all() and np.isnan(stored[4, cells - 8:]).all()
    assert red[-1] == 16 == np.count_nonzero(~np.isfinite(stored))


def test_checkpoint_resume_is_bitwise(gpu_lib):
    lee = gpu_lib
    name, shape = "D3Q7", (128, 16, 12)
    cells = int(np.prod(shape))
    rho, u, th = inputs.random_fields(shape, 3, 8)
    with lee.Solver(name, shape, 0.6, storage="bfp16") as a:
        a.init_fields(rho, u, th)
        a.step(10)
        full = np.empty((7, cells))
        a.get_populations(full)
    with lee.Solver(name, shape, 0.6, storage="bfp16") as b:
        b.init_fields(rho, u, th)
        b.step(4)
        ck = np.empty((7, cells))
        b.get_populations(ck)
    with lee.Solver(name, shape, 0.6, storage="bfp16") as c:
        c.set_populations(ck)  # decoded values encode back to the same values
        c.step(6)
        resumed = np.empty((7, cells))
        c.get_populations(resumed)
    assert np.array_equal(full, resumed)
