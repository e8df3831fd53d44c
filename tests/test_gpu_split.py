"""Split storage (LEE_STORE_SPLIT16: FP32 moments + FP16 non-equilibrium parts, periodic grids)
against the FP64 oracle, and against plain FP16 storage on the same runs."""
import numpy as np
import pytest

import oracle
from paper_1601_08103_gb300 import inputs

from test_gpu_parity import perm_to_lib, rel_l2, run_pair, shapes_for

pytestmark = pytest.mark.gpu

SETS = ["D1Q3", "D2Q5", "D2Q5_DI", "D3Q7", "D3Q9", "D3Q13", "D3Q19", "D3Q7_DI"]


def pulse_fields(s, shape, width=3.0, amp=1e-3):
    cells = int(np.prod(shape))
    rho = inputs.gaussian_pulse(shape, amp, width, [n / 2.3 for n in shape])
    u, th = inputs.zero_rest(s.D, cells)
    return rho, u, th


@pytest.mark.parametrize("name", SETS)
@pytest.mark.parametrize("vector", [True, False])
def test_split_storage_matches_oracle_and_beats_fp16(gpu_lib, name, vector):
    """Only the non-equilibrium part is rounded to 16 bits, so the error stays far below plain
    FP16 storage's, within the same FP16 bound."""
    s = oracle.velset(name)
    shape = shapes_for(s.D, vector)[0]
    n = 40
    f = pulse_fields(s, shape)
    r = run_pair(gpu_lib, name, shape, 0.55, n, storage="split16", fields=f)
    r16 = run_pair(gpu_lib, name, shape, 0.55, n, storage="f16", fields=f)
    bound = 4 * 2.0 ** -11 * np.sqrt(10 * n)
    err = rel_l2(r["m_gpu"][0], r["m_ora"][0])
    err16 = rel_l2(r16["m_gpu"][0], r16["m_ora"][0])
    assert err <= bound, (err, bound)
    assert err <= err16 / 4, (err, err16)
    errg = rel_l2(r["g_gpu"], r["g_ora"])
    assert errg <= bound, errg
    for a in range(s.D):
        assert rel_l2(r["m_gpu"][1][a], r["m_ora"][1][a]) <= bound


@pytest.mark.parametrize("name", ["D2Q5", "D3Q19"])
def test_split_reduction_and_conservation(gpu_lib, name):
    """The reduction sums the populations the state encodes (as exported) like the oracle does,
    and mass, momentum and energy stay conserved up to the rounding of the stored parts."""
    lee = gpu_lib
    s = oracle.velset(name)
    shape = shapes_for(s.D, True)[0]
    cells = int(np.prod(shape))
    rho, u, th = inputs.random_fields(shape, s.D, 5)
    p = perm_to_lib(lee, name)
    with lee.Solver(name, shape, 0.6, storage="split16") as sv:
        sv.init_fields(rho, u, th)
        red0 = np.empty(s.D + 4)
        sv.reduce(red0)
        sv.step(30)
        g = np.empty((s.q, cells))
        sv.get_populations(g)
        red = np.empty(s.D + 4)
        sv.reduce(red)
    want = oracle.reduce(name, g[np.argsort(p)])
    np.testing.assert_allclose(red[:-1], want[:-1], rtol=1e-12, atol=1e-15 * np.abs(g).sum())
    assert red[-1] == 0
    # the FP16 rounding of n* (relative 2^-11) does not keep its moments exactly zero: a random
    # walk over cells and steps, far below 2^-11 of the total
    scale = np.abs(g).sum()
    np.testing.assert_allclose(red[: s.D + 2], red0[: s.D + 2], atol=2e-5 * scale)


def test_split_checkpoint_round_trip(gpu_lib):
    """Export to FP64 and import again: the re-encoded state reproduces the populations to the
    rounding of its parts (the FP16 non-equilibrium part has moments of 2^-11 of its size, which
    the import folds into the FP32 moments and rounds again), and the run continues from it."""
    lee = gpu_lib
    name, shape = "D3Q19", (36, 10, 7)
    s = oracle.velset(name)
    cells = int(np.prod(shape))
    rho, u, th = pulse_fields(s, shape)
    with lee.Solver(name, shape, 0.6, storage="split16") as a:
        a.init_fields(rho, u, th)
        a.step(6)
        g1 = np.empty((s.q, cells))
        a.get_populations(g1)
        scale = a.store_scale
        a.step(5)
        full = np.empty((s.q, cells))
        a.get_populations(full)
    with lee.Solver(name, shape, 0.6, storage="split16", store_scale=scale) as b:
        b.set_populations(g1)
        g2 = np.empty((s.q, cells))
        b.get_populations(g2)
        assert rel_l2(g2, g1) < 5e-5
        b.step(5)
        resumed = np.empty((s.q, cells))
        b.get_populations(resumed)
    assert rel_l2(resumed, full) < 1e-4


@pytest.mark.parametrize("name,shape", [("D3Q19", (128, 9, 6)), ("D3Q13", (128, 6, 5)), ("D2Q5", (256, 10, 1)),
                                        ("D1Q3", (1024, 1, 1)), ("D3Q19", (64, 2, 3)), ("D3Q19", (192, 5, 1)),
                                        ("D3Q19", (64, 3, 2)), ("D3Q7", (256, 7, 4)), ("D3Q9", (128, 4, 3)),
                                        ("D3Q19", (64, 13, 11))])
def test_split_tiled_vector_and_scalar_paths_agree_bitwise(gpu_lib, monkeypatch, name, shape):
    """Grids whose width is a multiple of 32 V run the y-tiled vector kernel (the last tile row
    partly empty, and grids of 1-3 rows or planes whose source rows wrap onto themselves, here);
    it computes every cell with the same arithmetic as the one-cell-per-thread kernel, so the
    states agree bit for bit, and both match the oracle."""
    lee = gpu_lib
    s = oracle.velset(name)
    cells = int(np.prod(shape))
    f = pulse_fields(s, shape, width=4.0)
    outs = []
    for scalar in (False, True):
        monkeypatch.setenv("LEE_FORCE_SCALAR", "1" if scalar else "0")
        with lee.Solver(name, shape, 0.55, storage="split16", store_scale=1024.0) as sv:
            sv.init_fields(*f)
            sv.step(7)
            g = np.empty((s.q, cells))
            sv.get_populations(g)
            outs.append(g)
    assert np.array_equal(outs[0], outs[1])
    r = run_pair(lee, name, shape, 0.55, 7, storage="split16", fields=f)
    assert rel_l2(r["m_gpu"][0], r["m_ora"][0]) <= 4 * 2.0 ** -11 * np.sqrt(70)
