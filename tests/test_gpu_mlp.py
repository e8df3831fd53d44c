"""Boundary network on the GPU (include/lee_mlp.h) against the FP64 oracle (oracle/mlp.py).

Both sides round the weights and every GEMM input to BF16; the GPU accumulates in FP32 and
evaluates GELU in FP32, the oracle in FP64.  Tolerances: forward rel L2 1e-4 (an FP32 pre-
activation can land on the other side of a BF16 rounding boundary for a handful of elements);
gradients rel L2 3e-3 per tensor (the same effect on the BF16-rounded back-propagated operands,
summed over rows).
"""
import numpy as np
import pytest

import oracle
from oracle import mlp as omlp
from paper_1601_08103_gb300 import inputs

pytestmark = pytest.mark.gpu


def _cuda(a, dtype=None):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a)).to(dtype or torch.float32).cuda()


def test_forward_matches_oracle(gpu_lib):
    import torch

    lee = gpu_lib
    p = omlp.init_params(1)
    rng = np.random.default_rng(2)
    rows = 1000  # 15 full 64-row blocks and a ragged tail
    x = rng.normal(size=(rows, 16)).astype(np.float32)
    x[:, 15] = 0
    with lee.Mlp(p.astype(np.float32)) as m:
        y = torch.empty(rows, device="cuda")
        m.forward(_cuda(x), rows, y)
        torch.cuda.synchronize()
    want, _ = omlp.forward(p, x.astype(np.float64))
    got = y.cpu().numpy().astype(np.float64)
    assert np.linalg.norm(got - want) / np.linalg.norm(want) < 1e-4


@pytest.mark.parametrize("rows", [64, 1000, 20000])
def test_loss_and_gradient_match_oracle(gpu_lib, rows):
    import torch

    lee = gpu_lib
    p = omlp.init_params(3)
    rng = np.random.default_rng(rows)
    x = rng.normal(size=(rows, 16)).astype(np.float32)
    x[:, 15] = 0
    t = rng.normal(size=rows).astype(np.float32)
    with lee.Mlp(p.astype(np.float32)) as m:
        grad = torch.empty(lee.MLP_NPARAM, device="cuda")
        loss = torch.empty(1, device="cuda")
        m.loss_grad(_cuda(x), _cuda(t), rows, grad, loss)
        torch.cuda.synchronize()
    L, g = omlp.loss_and_grad(p, x.astype(np.float64), t.astype(np.float64))
    assert float(loss.item()) == pytest.approx(L, rel=1e-4)
    gg = grad.cpu().numpy().astype(np.float64)
    for name, (a, b) in {"W1": (0, 1024), "b1": (1024, 1088), "W2": (1088, 5184), "b2": (5184, 5248),
                         "W3": (5248, 5312), "b3": (5312, 5313)}.items():
        err = np.linalg.norm(gg[a:b] - g[a:b]) / max(np.linalg.norm(g[a:b]), 1e-30)
        assert err < 3e-3, (name, err)


def test_gradient_is_deterministic(gpu_lib):
    import torch

    lee = gpu_lib
    p = omlp.init_params(4).astype(np.float32)
    rng = np.random.default_rng(5)
    x = _cuda(rng.normal(size=(5000, 16)))
    t = _cuda(rng.normal(size=5000))
    outs = []
    for _ in range(2):
        with lee.Mlp(p) as m:
            grad = torch.empty(lee.MLP_NPARAM, device="cuda")
            m.loss_grad(x, t, 5000, grad)
            torch.cuda.synchronize()
            outs.append(grad.cpu().numpy())
    assert np.array_equal(outs[0], outs[1])


def test_adam_step_moves_each_parameter_by_the_learning_rate(gpu_lib):
    """First Adam step: p - lr * g / |g| (bias correction makes m_hat = g, v_hat = g^2), checked
    on the parameters whose oracle gradient is clearly non-zero."""
    import torch

    lee = gpu_lib
    p = omlp.init_params(6)
    rng = np.random.default_rng(7)
    rows = 4096
    x = rng.normal(size=(rows, 16)).astype(np.float32)
    x[:, 15] = 0
    t = rng.normal(size=rows).astype(np.float32)
    lr = 1e-3
    with lee.Mlp(p.astype(np.float32)) as m:
        m.loss_grad(_cuda(x), _cuda(t), rows)
        m.adam_step(lr, 0.9, 0.999, 1e-12)
        after = np.empty(lee.MLP_NPARAM, dtype=np.float32)
        m.get_params(after)
    _, g = omlp.loss_and_grad(p, x.astype(np.float64), t.astype(np.float64))
    want, _, _ = omlp.adam_step(p, np.zeros_like(p), np.zeros_like(p), g, 1, lr, eps=1e-12)
    sel = np.abs(g) > 1e-2 * np.abs(g).max()
    assert sel.sum() > 1000
    np.testing.assert_allclose(after[sel], want[sel], atol=2e-7)


def test_training_reduces_the_loss(gpu_lib):
    """A learnable target (a fixed linear map of the inputs through tanh) is fitted by the GPU's
    forward, backward and Adam kernels alone."""
    import torch

    lee = gpu_lib
    rng = np.random.default_rng(8)
    rows = 8192
    x = rng.normal(size=(rows, 16)).astype(np.float32)
    x[:, 15] = 0
    w = rng.normal(size=16) / 4
    t = np.tanh(x @ w).astype(np.float32)
    xd, td = _cuda(x), _cuda(t)
    loss = torch.empty(1, device="cuda")
    hist = []
    with lee.Mlp(omlp.init_params(9).astype(np.float32)) as m:
        for it in range(300):
            m.loss_grad(xd, td, rows, None, loss)
            m.adam_step(3e-3)
            if it % 50 == 0 or it == 299:
                hist.append(float(loss.item()))
    assert hist[-1] < 0.05 * hist[0], hist


def _open_state(lee, storage, nx, ny, seed):
    s = oracle.velset("D2Q5")
    rng = np.random.default_rng(seed)
    g = 1e-3 * rng.normal(size=(5, nx * ny))
    return s, g


def test_edge_inputs_match_oracle_strips(gpu_lib):
    import torch

    lee = gpu_lib
    nx, ny = 37, 21
    s, g = _open_state(lee, "f64", nx, ny, 3)
    lib_c = lee.lee_velset_info("D2Q5")["c"]
    idx = {tuple(int(v) for v in c): j for j, c in enumerate(s.c)}
    perm = [idx[tuple(c)] for c in lib_c]
    for storage in ("f64", "f32"):
        with lee.Solver("D2Q5", (nx, ny, 1), 0.6, storage=storage, bc="open_zero") as sv:
            sv.set_populations(g[perm])
            R = 2 * (nx + ny)
            xd = torch.empty((R, 16), device="cuda")
            sd = torch.empty(R, device="cuda")
            lee.lee_lbm_edge_inputs(sv.h, xd, sd)
            torch.cuda.synchronize()
        X, S, E, P = omlp.strips(g, (nx, ny, 1), s.c, s.f, (0, 0, nx, ny))
        np.testing.assert_allclose(xd.cpu().numpy(), X, atol=2e-6)
        np.testing.assert_allclose(sd.cpu().numpy(), S, rtol=2e-6)


def test_batch_edge_samples_match_oracle(gpu_lib):
    import torch

    lee = gpu_lib
    doms = [(40, 30, 0.6), (48, 36, 0.7), (40, 40, 0.9)]
    region = (5, 4, 20, 17)
    fields = [inputs.random_fields((nx, ny, 1), 2, 11 + d) for d, (nx, ny, _) in enumerate(doms)]
    with lee.Batch("D2Q5", "f32", doms) as b:
        for d, f in enumerate(fields):
            b.init_fields(d, *f)
        b.step(9, "sequential")
        R = 2 * (region[2] + region[3])
        xd = torch.empty((3 * R, 16), device="cuda")
        td = torch.empty(3 * R, device="cuda")
        sd = torch.empty(3 * R, device="cuda")
        lee.lee_batch_edge_samples(b.b, *region, xd, td, sd)
        posts = []
        for d, (nx, ny, _) in enumerate(doms):
            gp = np.empty((5, nx * ny))
            b.get_populations(d, gp)
            posts.append(gp)
        torch.cuda.synchronize()
    s = oracle.velset("D2Q5")
    lib_c = lee.lee_velset_info("D2Q5")["c"]
    for d, (nx, ny, _) in enumerate(doms):
        # the oracle reads the same populations, given in the library's velocity order
        X, S, _, _ = omlp.strips(posts[d], (nx, ny, 1), np.array(lib_c), np.array(lee.lee_velset_info("D2Q5")["f"]),
                                 region)
        T = omlp.targets(posts[d], (nx, ny, 1), np.array(lib_c), np.array(lee.lee_velset_info("D2Q5")["f"]), region)
        sl = slice(d * R, (d + 1) * R)
        np.testing.assert_allclose(xd.cpu().numpy()[sl], X, atol=2e-6)
        np.testing.assert_allclose(td.cpu().numpy()[sl], T, rtol=2e-5, atol=2e-6)
        np.testing.assert_allclose(sd.cpu().numpy()[sl], S, rtol=2e-6)


@pytest.mark.parametrize("storage", ["f64", "f32"])
def test_learned_boundary_step_matches_oracle(gpu_lib, storage):
    """Every step: network on the edge strips of the post-collision state -> entering
    populations -> open step; the oracle runs the same loop with its FP64 network."""
    lee = gpu_lib
    nx, ny, tau, n = 48, 33, 0.6, 12
    s = oracle.velset("D2Q5")
    c = [n_ / 2.5 for n_ in (nx, ny, 1)]
    rho = inputs.gaussian_pulse((nx, ny, 1), 1e-3, 6.0, c, periodic=False)
    u, th = inputs.zero_rest(2, nx * ny)
    p = omlp.init_params(12) * 0.5
    with lee.Solver("D2Q5", (nx, ny, 1), tau, storage=storage, bc="open_learned") as sv:
        sv.set_boundary_mlp(p.astype(np.float32))
        sv.init_fields(rho, u, th)
        sv.step(n)
        r_gpu = np.empty(nx * ny)
        sv.moments(r_gpu)
    g = oracle.equilibrium("D2Q5", rho, u, th)
    for _ in range(n):
        post = oracle.post_state("D2Q5", (nx, ny, 1), tau, g, bc="open_zero")
        ghost = omlp.ghost_values(p, post, (nx, ny, 1), s.c, s.f)
        g = oracle.step("D2Q5", (nx, ny, 1), tau, g, 1, bc="open_ghost", ghost=ghost)
    r_ora = oracle.moments("D2Q5", g)[0]
    err = np.linalg.norm(r_gpu - r_ora) / np.linalg.norm(r_ora)
    assert err < (1e-5 if storage == "f64" else 3e-5), err


@pytest.mark.parametrize("storage", ["f16", "bf16"])
def test_learned_boundary_16bit_storage_against_oracle(gpu_lib, storage):
    """The learned step on 16-bit storage (scaled values, FP32 network and collision) against the
    oracle's FP64 loop, 24 steps.  Every step rounds each stored population once to 16 bits
    (relative error at most 2^-11 for FP16, 2^-8 for BF16); the bound allows twice that times
    sqrt(n).  For FP16 the bound is also well below what the edge changes: the same run with
    zero-incoming edges differs from the learned one by more than three times the bound."""
    lee = gpu_lib
    nx, ny, tau, n = 48, 33, 0.6, 24
    s = oracle.velset("D2Q5")
    c = [n_ / 2.5 for n_ in (nx, ny, 1)]
    rho = inputs.gaussian_pulse((nx, ny, 1), 1e-3, 6.0, c, periodic=False)
    u, th = inputs.zero_rest(2, nx * ny)
    p = omlp.init_params(12) * 0.5
    with lee.Solver("D2Q5", (nx, ny, 1), tau, storage=storage, bc="open_learned") as sv:
        sv.set_boundary_mlp(p.astype(np.float32))
        sv.init_fields(rho, u, th)
        sv.step(n)
        r_gpu = np.empty(nx * ny)
        sv.moments(r_gpu)
    g = oracle.equilibrium("D2Q5", rho, u, th)
    for _ in range(n):
        post = oracle.post_state("D2Q5", (nx, ny, 1), tau, g, bc="open_zero")
        ghost = omlp.ghost_values(p, post, (nx, ny, 1), s.c, s.f)
        g = oracle.step("D2Q5", (nx, ny, 1), tau, g, 1, bc="open_ghost", ghost=ghost)
    r_ora = oracle.moments("D2Q5", g)[0]
    unit = 2.0 ** -11 if storage == "f16" else 2.0 ** -8
    bound = 2 * unit * np.sqrt(n)
    err = np.linalg.norm(r_gpu - r_ora) / np.linalg.norm(r_ora)
    assert 0 < err < bound, (err, bound)
    if storage == "f16":
        gz = oracle.step("D2Q5", (nx, ny, 1), tau, oracle.equilibrium("D2Q5", rho, u, th), n, bc="open_zero")
        edge = np.linalg.norm(oracle.moments("D2Q5", gz)[0] - r_ora) / np.linalg.norm(r_ora)
        assert edge > 3 * bound, (edge, bound)


def _learned_run(lee, monkeypatch, env, name, shape, storage, params, fields, calls):
    for k in ("LEE_LEARNED_STREAMS", "LEE_FORCE_SCALAR"):
        monkeypatch.delenv(k, raising=False)
    for k, v in env.items():
        monkeypatch.setenv(k, v)
    q = lee.lee_velset_info(name)["q"]
    with lee.Solver(name, shape, 0.6, storage=storage, bc="open_learned") as sv:
        sv.set_boundary_mlp(params)
        sv.init_fields(*fields)
        for n in calls:
            sv.step(n)
        g = np.empty((q, int(np.prod(shape))))
        sv.get_populations(g)
    return g


LEARNED_SHAPES = [(48, 33, 1), (64, 64, 1), (3, 3, 1), (5, 4, 1), (7, 130, 1), (130, 7, 1), (257, 19, 1),
                  (2048, 2048, 1), (4100, 12, 1)]


@pytest.mark.parametrize("storage", ["f64", "f32", "f16", "bf16"])
@pytest.mark.parametrize("shape", LEARNED_SHAPES)
def test_one_launch_learned_step_equals_three_launch_form(gpu_lib, monkeypatch, storage, shape):
    """k_learned_step (network blocks that also write their border cells, corner cells completed by
    the second of their two rows, interior blocks) against the network kernel + k_edge_fixup on a
    side stream and the interior step (LEE_LEARNED_STREAMS=1): equal bit for bit, through a
    captured graph (10 steps), direct launches (3, then 1) and another graph (8), so the corner
    counters cross launches of both kinds.  Shapes cover grids with fewer than 16 border rows,
    border rows not a multiple of 16, widths that take the one-cell-per-thread interior, and a
    2048^2 grid (1024 network blocks beside 4096 interior blocks)."""
    lee = gpu_lib
    D = 2
    params = (omlp.init_params(31) * 0.5).astype(np.float32)
    fields = inputs.random_fields(shape, D, 41)
    calls = (10, 3, 1, 8)
    g1 = _learned_run(lee, monkeypatch, {}, "D2Q5", shape, storage, params, fields, calls)
    g3 = _learned_run(lee, monkeypatch, {"LEE_LEARNED_STREAMS": "1"}, "D2Q5", shape, storage, params, fields, calls)
    assert np.isfinite(g1).all()
    assert np.array_equal(g1, g3)


@pytest.mark.parametrize("storage", ["f32", "f16"])
def test_one_launch_learned_step_scalar_interior(gpu_lib, monkeypatch, storage):
    """LEE_FORCE_SCALAR=1 (one cell per interior thread) gives the same state as the vector form."""
    lee = gpu_lib
    shape = (64, 40, 1)
    params = (omlp.init_params(32) * 0.5).astype(np.float32)
    fields = inputs.random_fields(shape, 2, 43)
    g_v = _learned_run(lee, monkeypatch, {}, "D2Q5", shape, storage, params, fields, (9,))
    g_s = _learned_run(lee, monkeypatch, {"LEE_FORCE_SCALAR": "1"}, "D2Q5", shape, storage, params, fields, (9,))
    assert np.array_equal(g_v, g_s)
