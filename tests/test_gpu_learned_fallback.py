"""The learned edge's fallback (include/lee_lbm.h, LEE_BC_OPEN_LEARNED): without an installed
network -- or with one trained for another tau -- the grid runs the plain buffer, the configured
sponge frame (zero-incoming edges if its width is 0), bit for bit like an OPEN_SPONGE (OPEN_ZERO)
handle and within 1e-12 of the oracle's sponge in FP64; installing a network switches to the
learned edge, also after graphs of the fallback were captured."""
import numpy as np
import pytest

from paper_1601_08103_gb300 import inputs

from test_gpu_parity import assert_close, run_pair

pytestmark = pytest.mark.gpu

SHAPE = (64, 48, 1)


def _run(lee, bc, storage, n, fields, params=None, trained_tau=None, tau=0.6, w=4, smax=0.5):
    with lee.Solver("D2Q5", SHAPE, tau, storage=storage, bc=bc, sponge_width=w, sponge_strength=smax) as sv:
        installed = None
        if params is not None:
            installed = sv.set_boundary_mlp_for_tau(params, trained_tau)
        mode = sv.boundary_in_use
        sv.init_fields(*fields)
        sv.step(n)
        g = np.empty((5, SHAPE[0] * SHAPE[1]))
        sv.get_populations(g)
    return g, mode, installed


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_no_network_runs_the_sponge_frame(gpu_lib, storage):
    lee = gpu_lib
    fields = inputs.random_fields(SHAPE, 2, 3)
    for n in (1, 9):
        got, mode, _ = _run(lee, "open_learned", storage, n, fields)
        want, _, _ = _run(lee, "open_sponge", storage, n, fields)
        assert mode == "open_sponge"
        assert np.array_equal(got, want)
        got0, mode0, _ = _run(lee, "open_learned", storage, n, fields, w=0, smax=0.0)
        want0, _, _ = _run(lee, "open_zero", storage, n, fields, w=0, smax=0.0)
        assert mode0 == "open_zero" and np.array_equal(got0, want0)
    if storage == "f64":  # and the sponge frame is the oracle's
        r = run_pair(lee, "D2Q5", SHAPE, 0.6, 9, storage="f64", bc="open_sponge", fields=fields, sponge_w=4, smax=0.5)
        assert_close(got, r["g_ora"], 1e-12, "fallback sponge vs oracle")


def test_network_for_another_tau_is_not_installed(gpu_lib):
    from oracle import mlp as omlp

    lee = gpu_lib
    params = omlp.init_params(3).astype(np.float32)
    fields = inputs.random_fields(SHAPE, 2, 4)
    got, mode, installed = _run(lee, "open_learned", "f32", 9, fields, params=params, trained_tau=0.6, tau=0.7)
    want, _, _ = _run(lee, "open_sponge", "f32", 9, fields, tau=0.7)
    assert installed is False and mode == "open_sponge" and np.array_equal(got, want)
    got2, mode2, installed2 = _run(lee, "open_learned", "f32", 9, fields, params=params, trained_tau=0.6, tau=0.6)
    assert installed2 is True and mode2 == "open_learned"
    with lee.Solver("D2Q5", SHAPE, 0.6, storage="f32", bc="open_learned") as sv:  # the plain install
        sv.set_boundary_mlp(params)
        sv.init_fields(*fields)
        sv.step(9)
        ref = np.empty_like(got2)
        sv.get_populations(ref)
    assert np.array_equal(got2, ref)


def test_installing_a_network_after_fallback_steps(gpu_lib):
    """Graphs captured while the fallback ran are dropped when the network arrives."""
    from oracle import mlp as omlp

    lee = gpu_lib
    params = omlp.init_params(5).astype(np.float32)
    fields = inputs.random_fields(SHAPE, 2, 6)
    cells = SHAPE[0] * SHAPE[1]
    with lee.Solver("D2Q5", SHAPE, 0.6, storage="f32", bc="open_learned", sponge_width=4, sponge_strength=0.5) as a:
        a.init_fields(*fields)
        a.step(9)
        mid = np.empty((5, cells))
        a.get_populations(mid)
        a.set_boundary_mlp(params)
        assert a.boundary_in_use == "open_learned"
        a.step(9)
        got = np.empty((5, cells))
        a.get_populations(got)
    with lee.Solver("D2Q5", SHAPE, 0.6, storage="f32", bc="open_sponge", sponge_width=4, sponge_strength=0.5) as b:
        b.init_fields(*fields)
        b.step(9)
        ref_mid = np.empty((5, cells))
        b.get_populations(ref_mid)
    assert np.array_equal(mid, ref_mid)
    with lee.Solver("D2Q5", SHAPE, 0.6, storage="f32", bc="open_learned") as c:
        c.set_boundary_mlp(params)
        c.set_populations(mid)
        c.step(9)
        want = np.empty((5, cells))
        c.get_populations(want)
    assert np.array_equal(got, want)
