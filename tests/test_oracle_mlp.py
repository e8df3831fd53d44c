"""Pins of the boundary-network oracle (oracle/mlp.py): BF16 rounding against torch's conversion,
the backward pass against central finite differences, Adam's closed-form first step, the GELU's
known values, and the edge-strip geometry against rotations of the grid."""
import math

import numpy as np
import pytest

import oracle
from oracle import mlp


def test_bf16_rounding_matches_torch():
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(0)
    x = np.concatenate([rng.normal(size=5000) * 10.0 ** rng.integers(-8, 8, size=5000),
                        np.array([1.0 + 2.0 ** -8, 1.0 + 3 * 2.0 ** -8, -(1.0 + 2.0 ** -8), 0.0, -0.0, 65504.0])])
    want = torch.tensor(x, dtype=torch.float32).to(torch.bfloat16).to(torch.float64).numpy()
    np.testing.assert_array_equal(mlp.bf16(x), want)


def test_gelu_known_values():
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert mlp.gelu_grad(np.array([0.0]))[0] == pytest.approx(0.5, abs=1e-15)
    z = np.array([8.0, -8.0])
    np.testing.assert_allclose(mlp.gelu(z), [8.0, 0.0], atol=1e-13)
    # GELU(1) = Phi(1) = (1 + erf(1/sqrt 2)) / 2
    assert mlp.gelu(np.array([1.0]))[0] == pytest.approx(0.8413447460685429, abs=1e-15)


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(1)
    p = mlp.init_params(3) + 0.01 * rng.normal(size=mlp.NPARAM)
    x = rng.normal(size=(9, 16))
    t = rng.normal(size=9)
    L, g = mlp.loss_and_grad(p, x, t, quantize=False)
    idx = rng.choice(mlp.NPARAM, 60, replace=False)
    idx = np.concatenate([idx, [mlp.NPARAM - 1, 1024, 1088, 5248]])  # b3, b1[0], W2[0][0], W3[0]
    h = 1e-6
    for i in idx:
        e = np.zeros(mlp.NPARAM)
        e[i] = h
        fd = (mlp.loss_and_grad(p + e, x, t, quantize=False)[0] - mlp.loss_and_grad(p - e, x, t, quantize=False)[0]) / (2 * h)
        assert g[i] == pytest.approx(fd, rel=1e-5, abs=1e-9), i


def test_quantized_gradient_is_close_to_exact():
    rng = np.random.default_rng(2)
    p = mlp.init_params(4)
    x = rng.normal(size=(256, 16))
    x[:, 15] = 0
    t = rng.normal(size=256)
    _, gq = mlp.loss_and_grad(p, x, t, quantize=True)
    _, ge = mlp.loss_and_grad(p, x, t, quantize=False)
    assert np.linalg.norm(gq - ge) / np.linalg.norm(ge) < 2e-2


def test_adam_first_step_is_signed_learning_rate():
    rng = np.random.default_rng(3)
    p = rng.normal(size=50)
    g = rng.normal(size=50)
    p1, m, v = mlp.adam_step(p, np.zeros(50), np.zeros(50), g, 1, lr=1e-3, eps=0.0)
    np.testing.assert_allclose(p1, p - 1e-3 * np.sign(g), atol=1e-15)


def test_constant_network_gives_closed_form_ghosts():
    s = oracle.velset("D2Q5")
    nx, ny = 30, 25
    rng = np.random.default_rng(5)
    post = rng.normal(size=(5, nx * ny))
    d = mlp.unpack(np.zeros(mlp.NPARAM))
    d["b3"] = np.array([1.0])  # exactly representable
    p = mlp.pack(d)
    ghost = mlp.ghost_values(p, post, (nx, ny, 1), s.c, s.f)
    X, S, E, P = mlp.strips(post, (nx, ny, 1), s.c, s.f, (0, 0, nx, ny))
    f_in = 0.125  # every entering velocity is a moving one
    scaled = 0
    for g0 in range(0, len(S), 16):
        sl = slice(g0, g0 + 16)
        vin = 1.0 * S[sl]
        hout = X[sl, 2] * S[sl]
        a = min(1.0, np.sqrt(np.sum(hout ** 2) / np.sum(vin ** 2)))
        scaled += a < 1.0
        for v, e, k in zip(vin, E[sl], P[sl]):
            assert ghost[e, k] == pytest.approx(a * v * f_in, rel=1e-14)
    assert 0 < scaled < (len(S) + 15) // 16  # both branches of the bound are exercised
    # the inputs have unit rms
    np.testing.assert_allclose(np.sqrt(np.mean(X[:, :15] ** 2, axis=1)), 1.0, rtol=1e-12)
    assert np.all(X[:, 15] == 0)


def _rotate_quarter(post, n, c):
    """Rotate a D2Q5 field on an n x n grid by +90 degrees: cell (x, y) -> (n-1-y, x), velocity
    (cx, cy) -> (-cy, cx)."""
    idx = {(int(v[0]), int(v[1])): i for i, v in enumerate(c)}
    out = np.empty_like(post)
    for i, v in enumerate(c):
        j = idx[(-int(v[1]), int(v[0]))]
        f = post[i].reshape(n, n)  # [y][x]
        rot = np.empty_like(f)
        for y in range(n):
            for x in range(n):
                rot[x, n - 1 - y] = f[y, x]
        out[j] = rot.ravel()
    return out


def test_strips_and_targets_rotate_with_the_grid():
    """A proper rotation of the field maps each edge's strips (and targets) onto those of the
    rotated edge: left -> bottom, bottom -> right, right -> top, top -> left."""
    s = oracle.velset("D2Q5")
    n = 10
    rng = np.random.default_rng(7)
    post = rng.normal(size=(5, n * n))
    rot = _rotate_quarter(post, n, s.c)
    region = (1, 1, n - 2, n - 2)
    X0, S0, E0, P0 = mlp.strips(post, (n, n, 1), s.c, s.f, region)
    T0 = mlp.targets(post, (n, n, 1), s.c, s.f, region)
    X1, S1, E1, P1 = mlp.strips(rot, (n, n, 1), s.c, s.f, region)
    T1 = mlp.targets(rot, (n, n, 1), s.c, s.f, region)
    m = n - 2
    # cell (x, y) -> (n-1-y, x): left edge x = 1 at y -> bottom edge y = 1 at x = n-1-y (reversed
    # order along the edge); bottom edge (x, 1) -> right edge x = n-2 at y = x (same order)
    for k in range(m):
        a = 0 * m + k                 # left edge, position k (y = 1 + k)
        b = 2 * m + (m - 1 - k)       # bottom edge of the rotated field
        np.testing.assert_allclose(X1[b], X0[a], atol=1e-15)
        assert T1[b] == pytest.approx(T0[a], abs=1e-15)
        a = 2 * m + k                 # bottom edge, position k (x = 1 + k)
        b = 1 * m + k                 # right edge of the rotated field
        np.testing.assert_allclose(X1[b], X0[a], atol=1e-15)
        assert T1[b] == pytest.approx(T0[a], abs=1e-15)


def test_targets_are_the_streamed_in_values_of_a_periodic_grid():
    """On a periodic grid with the region = the whole grid minus nothing, the target of an edge
    cell is what the periodic step streams into it: ghost-fed step with targets*s*f = periodic."""
    s = oracle.velset("D2Q5")
    nx, ny = 8, 6
    rng = np.random.default_rng(9)
    g = rng.normal(size=(5, nx * ny))
    tau = 0.7
    post = oracle.collide("D2Q5", tau, g)
    # embed the grid in a 1-cell periodic frame so that "outside" cells exist
    big = np.zeros((5, (nx + 2) * (ny + 2)))
    P = post.reshape(5, ny, nx)
    B = big.reshape(5, ny + 2, nx + 2)
    for yy in range(-1, ny + 1):
        for xx in range(-1, nx + 1):
            B[:, yy + 1, xx + 1] = P[:, yy % ny, xx % nx]
    region = (1, 1, nx, ny)
    X, S, E, Pk = mlp.strips(big, (nx + 2, ny + 2, 1), s.c, s.f, region)
    T = mlp.targets(big, (nx + 2, ny + 2, 1), s.c, s.f, region)
    L = max(nx, ny)
    ghost = np.zeros((4, L))
    idx = {(int(v[0]), int(v[1])): i for i, v in enumerate(s.c)}
    for tv, sc, e, k in zip(T, S, E, Pk):
        ghost[e, k] = tv * sc * s.f[idx[mlp.CANON[e][1]]]
    want = oracle.step("D2Q5", (nx, ny, 1), tau, g, 1)
    got = oracle.step("D2Q5", (nx, ny, 1), tau, g, 1, bc="open_ghost", ghost=ghost)
    np.testing.assert_allclose(got, want, atol=1e-14)


def test_bounded_learned_edge_never_adds_weighted_energy():
    """With the passivity bound, even a random (untrained, large) network cannot make the weighted
    energy grow on an open grid at tau >= 1/2: the edge injects at most what leaves."""
    s = oracle.velset("D2Q5")
    nx, ny = 14, 11
    rng = np.random.default_rng(13)
    g = rng.normal(size=(5, nx * ny))
    p = mlp.init_params(14) * 8.0  # deliberately wild weights
    for tau in (0.5, 0.6, 1.3):
        e_prev = oracle.reduce("D2Q5", oracle.post_state("D2Q5", (nx, ny, 1), tau, g))[4]
        gg = g
        for _ in range(25):
            post = oracle.post_state("D2Q5", (nx, ny, 1), tau, gg)
            ghost = mlp.ghost_values(p, post, (nx, ny, 1), s.c, s.f)
            gg = oracle.step("D2Q5", (nx, ny, 1), tau, gg, 1, bc="open_ghost", ghost=ghost)
            e = oracle.reduce("D2Q5", oracle.post_state("D2Q5", (nx, ny, 1), tau, gg))[4]
            assert e <= e_prev * (1 + 1e-12), (tau, e, e_prev)
            e_prev = e
