"""Batched 2D domains (include/lee_batch.h) on the GPU.

Per domain, the batched launch must give exactly what a single-domain solver gives (same
arithmetic, same coefficients), in every mode and launch shape; FP64 is also held to the oracle.
"""
import numpy as np
import pytest

import oracle
from paper_1601_08103_gb300 import inputs

pytestmark = pytest.mark.gpu

DOMAINS = [(64, 64, 0.6), (128, 32, 0.52), (192, 96, 1.2), (36, 20, 0.75), (100, 7, 0.5), (256, 128, 0.9), (8, 8, 0.66)]


def run_batch(lee, storage, domains, nsteps, mode, fields, tuning=None):
    outs = []
    with lee.Batch("D2Q5", storage, domains) as b:
        if tuning:
            b.set_tuning(*tuning)
        for d, (rho, u, th) in enumerate(fields):
            b.init_fields(d, rho, u, th)
        b.step(nsteps, mode)
        for d, (nx, ny, _) in enumerate(domains):
            g = np.empty((5, nx * ny))
            b.get_populations(d, g)
            outs.append(g)
    return outs


def run_single(lee, storage, domains, nsteps, fields):
    outs = []
    for (nx, ny, tau), (rho, u, th) in zip(domains, fields):
        with lee.Solver("D2Q5", (nx, ny, 1), tau, storage=storage) as sv:
            sv.init_fields(rho, u, th)
            sv.step(nsteps)
            g = np.empty((5, nx * ny))
            sv.get_populations(g)
            outs.append(g)
    return outs


def fields_for(domains, seed=0):
    return [inputs.random_fields((nx, ny, 1), 2, seed + d) for d, (nx, ny, _) in enumerate(domains)]


@pytest.mark.parametrize("storage", ["f32", "f64"])
def test_batched_modes_equal_single_domain_bitwise(gpu_lib, storage):
    lee = gpu_lib
    fields = fields_for(DOMAINS)
    for nsteps in (1, 37, 250):  # 250 = two graph replays of 100 steps + 50 direct launches
        want = run_single(lee, storage, DOMAINS, nsteps, fields)
        for mode in ("graph", "launch", "sequential"):
            got = run_batch(lee, storage, DOMAINS, nsteps, mode, fields)
            for d in range(len(DOMAINS)):
                assert np.array_equal(got[d], want[d]), (storage, nsteps, mode, d)


@pytest.mark.parametrize("fused", [1, 2, 3, 4])
def test_batched_fused_steps_equal_single_domain_bitwise(gpu_lib, monkeypatch, fused):
    """LEE_TB_STEPS at create time sets how many steps the batched FP32 kernel fuses per launch
    (four by default); every choice gives each domain the bits of single steps."""
    lee = gpu_lib
    fields = fields_for(DOMAINS, 5)
    want = run_single(lee, "f32", DOMAINS, 4 * fused + 3, fields)
    monkeypatch.setenv("LEE_TB_STEPS", str(fused))
    for mode in ("graph", "launch"):
        got = run_batch(lee, "f32", DOMAINS, 4 * fused + 3, mode, fields)
        for d in range(len(DOMAINS)):
            assert np.array_equal(got[d], want[d]), (fused, mode, d)


def test_every_launch_shape_gives_the_same_result(gpu_lib):
    lee = gpu_lib
    doms = [(nx, ny, t) for nx, ny, t in DOMAINS if nx % 4 == 0]
    fields = fields_for(doms, 10)
    ref = run_batch(lee, "f32", doms, 11, "launch", fields, tuning=(256, 4))
    for shape in [(128, 2), (128, 4), (256, 2), (512, 2), (512, 4)]:
        got = run_batch(lee, "f32", doms, 11, "launch", fields, tuning=shape)
        for a, b in zip(got, ref):
            assert np.array_equal(a, b), shape


def test_autotuning_leaves_the_state_unchanged(gpu_lib):
    lee = gpu_lib
    fields = fields_for(DOMAINS, 20)
    with lee.Batch("D2Q5", "f32", DOMAINS) as b:
        for d, f in enumerate(fields):
            b.init_fields(d, *f)
        b.step(3, "sequential")
        before = [np.empty((5, nx * ny)) for nx, ny, _ in DOMAINS]
        for d, g in enumerate(before):
            b.get_populations(d, g)
        threads, cpt = b.tune()
        assert threads in (128, 256, 512) and cpt in (1, 2, 4)
        for d, g in enumerate(before):
            now = np.empty_like(g)
            b.get_populations(d, now)
            assert np.array_equal(now, g)


def test_batched_f64_matches_oracle(gpu_lib):
    lee = gpu_lib
    fields = fields_for(DOMAINS, 30)
    got = run_batch(lee, "f64", DOMAINS, 23, "graph", fields)
    for d, ((nx, ny, tau), (rho, u, th)) in enumerate(zip(DOMAINS, fields)):
        g = oracle.step("D2Q5", (nx, ny, 1), tau, oracle.equilibrium("D2Q5", rho, u, th), 23)
        post = oracle.post_state("D2Q5", (nx, ny, 1), tau, g)
        lib_c = lee.lee_velset_info("D2Q5")["c"]
        idx = {tuple(int(v) for v in c): j for j, c in enumerate(oracle.velset("D2Q5").c)}
        want = post[[idx[tuple(c)] for c in lib_c]]
        err = np.linalg.norm(got[d] - want) / np.linalg.norm(want)
        assert err < 1e-12, (d, err)


def test_full_batched_workload(gpu_lib):
    """The batched configuration: 96 domains, sizes from {128, ..., 1024}^2, tau in [0.52, 1.2],
    1000 steps as graph replays; equal bit for bit to the sequential plain launches, conserving,
    and two sampled domains held to the oracle within the FP32 tolerance."""
    lee = gpu_lib
    specs = inputs.batched_2d_specs(96, seed=4)
    doms = [(s["nx"], s["ny"], s["tau"]) for s in specs]
    fields = [inputs.batched_2d_fields(s) for s in specs]
    results = {}
    for mode in ("graph", "sequential"):
        with lee.Batch("D2Q5", "f32", doms) as b:
            for d, f in enumerate(fields):
                b.init_fields(d, *f)
            b.step(1000, mode)
            out = []
            for d, (nx, ny, _) in enumerate(doms):
                r = np.empty(nx * ny)
                b.moments(d, r, None, None)
                out.append(r)
            red = np.empty(6)
            b.reduce(0, red)
            results[mode] = (out, red)
    for a, c in zip(results["graph"][0], results["sequential"][0]):
        assert np.array_equal(a, c)
    # mass of domain 0 conserved
    rho0 = fields[0][0]
    assert abs(results["graph"][1][0] - rho0.sum()) <= 1e-6 * np.abs(rho0).sum()
    order = np.argsort([nx * ny for nx, ny, _ in doms])
    for d in order[:2]:
        nx, ny, tau = doms[d]
        g = oracle.step("D2Q5", (nx, ny, 1), tau, oracle.equilibrium("D2Q5", *fields[d]), 1000)
        want = oracle.moments("D2Q5", g)[0]
        err = np.linalg.norm(results["graph"][0][d] - want) / np.linalg.norm(want)
        assert err < 5e-5, (d, err)


MIXES = [[(nx, ny, t) for nx, ny, t in DOMAINS if nx % 4 == 0],
         [(256, 256, 0.6), (512, 128, 0.9), (128, 384, 0.55), (1024, 64, 1.1), (64, 200, 0.7)]]


@pytest.mark.parametrize("mix", [0, 1])
def test_autotuner_picks_a_fused_shape_with_the_same_bits(gpu_lib, monkeypatch, mix):
    """The tuner sweeps the fused kernel (steps per launch x tile rows x tile order) on the batch
    itself; whatever it picks, and any hand-set shape, gives each domain the bits of single
    steps."""
    lee = gpu_lib
    monkeypatch.delenv("LEE_TB_STEPS", raising=False)
    monkeypatch.delenv("LEE_SINGLE_STEP", raising=False)
    doms = MIXES[mix]
    fields = fields_for(doms, 50 + mix)
    n = 37
    want = run_single(lee, "f32", doms, n, fields)
    with lee.Batch("D2Q5", "f32", doms) as b:
        for d, f in enumerate(fields):
            b.init_fields(d, *f)
        shape = b.tune_shape()
        assert shape["threads"] in (128, 256, 512) and shape["cells_per_thread"] in (2, 4)
        assert shape["steps_per_launch"] in (1, 2, 3, 4) and shape["us_per_step"] > 0
        if shape["steps_per_launch"] > 1:
            assert shape["tile_rows"] in (32, 48, 64, 96, 128) and shape["tile_order"] in (0, 1)
        b.step(n, "graph")
        for d, (nx, ny, _) in enumerate(doms):
            g = np.empty((5, nx * ny))
            b.get_populations(d, g)
            assert np.array_equal(g, want[d]), (mix, d, shape)
    for steps, rows, order in ((2, 32, 1), (3, 96, 0), (4, 128, 1), (1, 64, 0)):
        with lee.Batch("D2Q5", "f32", doms) as b:
            b.set_shape(256, 4, steps, rows, order)
            assert b.tune_shape()["steps_per_launch"] == steps
            for d, f in enumerate(fields):
                b.init_fields(d, *f)
            b.step(n, "launch")
            for d, (nx, ny, _) in enumerate(doms):
                g = np.empty((5, nx * ny))
                b.get_populations(d, g)
                assert np.array_equal(g, want[d]), (steps, rows, order, d)


def test_set_shape_rejects_bad_shapes(gpu_lib):
    lee = gpu_lib
    with lee.Batch("D2Q5", "f32", MIXES[1]) as b:
        for args in ((100, 4, 4, 64, 0), (256, 3, 4, 64, 0), (256, 4, 5, 64, 0), (256, 4, 4, 62, 0),
                     (256, 4, 4, 64, 2), (256, 4, 4, 2048, 0)):
            with pytest.raises(lee.LeeError) as e:
                b.set_shape(*args)
            assert e.value.status == lee.LEE_ERR_INVALID_ARGUMENT, args
    with lee.Batch("D2Q5", "f64", MIXES[1]) as b:  # no fused kernel for FP64 storage
        with pytest.raises(lee.LeeError):
            b.set_shape(256, 2, 4, 64, 0)
        b.set_shape(256, 2, 1, 64, 0)
