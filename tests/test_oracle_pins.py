"""Pins of the FP64 CPU oracle against what the paper and the mathematics fix.

Each test ties the oracle to something other than itself: the printed velocity-set tables
(tests/golden/velsets.json), closed-form Maxwellian moments, the printed linear form H(tau) of the
step (assembled independently of the oracle's moment/equilibrium code), the d'Alembert solution,
exact conservation, the weighted-L2 stability structure, Fourier eigenmodes of Gamma(k), and
second-order convergence towards the exact LEE solution at tau = 1/2.
"""
import json
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
from oracle import analysis as an

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "velsets.json")))
ALL_SETS = ["D1Q3", "D2Q5", "D2Q5_DI", "D3Q7", "D3Q9", "D3Q13", "D3Q19", "D3Q7_DI"]
MONO = ["D1Q3", "D2Q5", "D3Q7", "D3Q9", "D3Q13", "D3Q19"]
UNITARY = [s for s in ALL_SETS if s != "D3Q19"]  # Sec. 8: Gamma(1/2) unitary for these


def frac(v):
    return float(Fraction(v[0], v[1]))


def shell(c):
    return int(np.abs(c).sum())


def grid_shape(D, n=(5, 4, 3)):
    return tuple(list(n[:D]) + [1] * (3 - D))


# --------------------------------------------------------------------------------------------
# tables
# --------------------------------------------------------------------------------------------

@pytest.mark.parametrize("name", ALL_SETS)
def test_tables_match_printed_values(name):
    s = oracle.velset(name)
    g = GOLD[name]
    assert s.D == g["D"] and s.q == g["q"]
    if name == "D3Q7_DI":
        f1 = frac(g["f1"])
        assert s.rho0 == pytest.approx(42 / 5 * f1, abs=1e-15)
        want_w = {0: 12 / 5 * f1, 1: f1}
    elif "shell_weights" in g:
        assert s.rho0 == pytest.approx(frac(g["rho0"]), abs=1e-15)
        want_w = {int(k): frac(v) for k, v in g["shell_weights"].items()}
    else:
        assert s.rho0 == pytest.approx(frac(g["rho0"]), abs=1e-15)
        want_w = {int(k): frac(v) for k, v in GOLD["family3d"]["expected"][name].items()}
    assert s.theta0 == pytest.approx(frac(g["theta0"]), abs=1e-15)
    for i in range(s.q):
        assert s.f[i] == pytest.approx(want_w[shell(s.c[i])], abs=1e-15), (name, s.c[i])
    # every shell the paper keeps is present, with the full symmetric star of velocities
    counts = {0: 1, 1: 2 * s.D, 2: 2 * s.D * (s.D - 1), 3: 8}
    for sh in want_w:
        assert sum(shell(c) == sh for c in s.c) == counts[sh]
    if "shell_beta" in g:
        for i in range(s.q):
            assert s.beta[i] == pytest.approx(frac(g["shell_beta"][str(shell(s.c[i]))]), abs=1e-15)
        assert s.a1 == pytest.approx(1 / s.rho0, abs=1e-15)
        assert s.a2 == pytest.approx(frac(g["a2"]), abs=1e-14)
        assert s.c1 == 0.0
        assert s.gamma == pytest.approx(frac(g["gamma"]), abs=1e-15)
        if name == "D2Q5_DI":
            assert s.b == pytest.approx(1 / s.theta0, abs=1e-14)
            assert s.c2 == pytest.approx(5 / s.theta0, abs=1e-13)
        else:
            assert s.b == pytest.approx(frac(g["b"]), abs=1e-14)
            assert s.c2 == pytest.approx(frac(g["c2"]), abs=1e-13)
    # velocities are symmetric (Sec. 4: S is a finite symmetric set)
    vs = {tuple(c) for c in s.c}
    assert all(tuple(-np.array(c)) in vs for c in vs)


@pytest.mark.parametrize("name", MONO)
def test_similarity_conditions_against_closed_form_maxwellian(name):
    """Sec. 4: discrete moments of f* of 1, |v|^2/2, v_a v_b, |v|^2 v_a v_b / 2, |v|^4/4 equal the
    Maxwellian's, which are closed-form Gaussian integrals."""
    s = oracle.velset(name)
    m = an.maxwellian_moments(s.D, s.rho0, s.theta0)
    d = an.discrete_moments(s)
    assert d["one"] == pytest.approx(m["one"], abs=1e-15)
    assert d["half_v2"] == pytest.approx(m["half_v2"], abs=1e-15)
    assert d["quarter_v4"] == pytest.approx(m["quarter_v4"], abs=1e-15)
    np.testing.assert_allclose(d["vavb"], m["vavb_diag"] * np.eye(s.D), atol=1e-15)
    np.testing.assert_allclose(d["half_v2_vavb"], m["half_v2_vavb_diag"] * np.eye(s.D), atol=1e-15)


# --------------------------------------------------------------------------------------------
# equilibrium and moments
# --------------------------------------------------------------------------------------------

@pytest.mark.parametrize("name", ALL_SETS)
def test_equilibrium_carries_the_lee_fluxes(name):
    """The equilibrium must reproduce the LEE (Sec. 5): its moments are (rho', u', theta'), its
    momentum flux is p' I with p' = rho0 theta' + theta0 rho' (Sec. 2.1), its energy density is
    (rho0 theta' + theta0 rho') / (gamma - 1) and its energy flux gamma/(gamma-1) rho0 theta0 u'."""
    s = oracle.velset(name)
    rng = np.random.default_rng(11)
    n = 6
    rho, theta = rng.normal(size=n), rng.normal(size=n)
    u = rng.normal(size=(s.D, n))
    g = oracle.equilibrium(name, rho, u, theta)
    r2, u2, t2 = oracle.moments(name, g)
    np.testing.assert_allclose(r2, rho, atol=1e-13)
    np.testing.assert_allclose(u2, u, atol=1e-13)
    np.testing.assert_allclose(t2, theta, atol=1e-13)
    c = s.c[:, : s.D].astype(float)
    c2 = (c * c).sum(1)
    p = s.rho0 * theta + s.theta0 * rho
    flux = np.einsum("ia,ib,in->nab", c, c, g)
    np.testing.assert_allclose(flux, p[:, None, None] * np.eye(s.D)[None], atol=1e-13)
    w = 0.5 * (c2 + s.beta)
    np.testing.assert_allclose(w @ g, p / (s.gamma - 1), atol=1e-13)
    np.testing.assert_allclose(np.einsum("i,ia,in->an", w, c, g),
                               s.gamma / (s.gamma - 1) * s.rho0 * s.theta0 * u, atol=1e-12)


@pytest.mark.parametrize("name", ALL_SETS)
def test_h_matrix_is_relaxation_onto_a_projection(name):
    """Sec. 8.3.1: H(1) is the equilibrium in matrix form and a projection, of rank D + 2 (the
    conserved moments); H(tau) = (1 - 1/tau) I + (1/tau) H(1)."""
    s = oracle.velset(name)
    P = an.h_matrix(s, 1.0)
    np.testing.assert_allclose(P @ P, P, atol=1e-14)
    assert np.linalg.matrix_rank(P, tol=1e-10) == min(s.D + 2, s.q)
    for tau in (0.5, 0.6, 0.8, 1.7):
        np.testing.assert_allclose(an.h_matrix(s, tau), (1 - 1 / tau) * np.eye(s.q) + P / tau, atol=1e-14)


@pytest.mark.parametrize("name", ALL_SETS)
def test_oracle_collision_equals_printed_linear_form(name):
    """The oracle's moments -> equilibrium -> relaxation equals H(tau) g with H from the printed
    entrywise formula of Sec. 6 (different code path)."""
    s = oracle.velset(name)
    rng = np.random.default_rng(3)
    g = rng.normal(size=(s.q, 17))
    for tau in (0.5, 0.55, 0.8, 1.2):
        np.testing.assert_allclose(oracle.collide(name, tau, g), an.h_matrix(s, tau) @ g, atol=1e-13)


def test_d1q3_collision_is_identity_and_gamma_as_printed():
    """Sec. 8.1: Gamma(k) = diag(1, e^{ik}, e^{-ik}) for D1Q3, i.e. H = I (three velocities,
    three conserved moments) for every tau."""
    s = oracle.velset("D1Q3")
    for tau in (0.5, 0.8, 2.0):
        np.testing.assert_allclose(an.h_matrix(s, tau), np.eye(3), atol=1e-15)
    for k in np.linspace(-np.pi, np.pi, 9):
        G = an.gamma_symbol(s, 0.5, [k])
        # velocity order of the oracle: 0, -1, +1 (as printed: c1 = 0, c2 = -1, c3 = 1)
        np.testing.assert_allclose(G, np.diag([1, np.exp(1j * k), np.exp(-1j * k)]), atol=1e-15)


@pytest.mark.parametrize("name", UNITARY)
def test_gamma_unitary_at_tau_half(name):
    """Sec. 8: Gamma(k, tau = 1/2) is unitary for every set except D3Q19."""
    s = oracle.velset(name)
    ks = np.linspace(-np.pi, np.pi, 5)
    for kx in ks:
        for ky in (ks if s.D > 1 else [0.0]):
            for kz in (ks[::2] if s.D > 2 else [0.0]):
                G = an.gamma_symbol(s, 0.5, [kx, ky, kz][: s.D])
                np.testing.assert_allclose(G.conj().T @ G, np.eye(s.q), atol=1e-13)


def test_d3q19_stability_structure():
    """Sec. 8.3.1: with A0 = diag(3, 13 I6, 52 I12), A0 H(1/2) is symmetric, and the collision
    matrix H(1/2) - I has eigenvalues 0 (five times) and -2 (fourteen times)."""
    s = oracle.velset("D3Q19")
    a0 = {0: 3.0, 1: 13.0, 2: 52.0}
    A0 = np.diag([a0[shell(c)] for c in s.c])
    H = an.h_matrix(s, 0.5)
    np.testing.assert_allclose(A0 @ H, (A0 @ H).T, atol=1e-13)
    ev = np.sort(np.linalg.eigvals(H - np.eye(19)).real)
    np.testing.assert_allclose(ev, [-2.0] * 14 + [0.0] * 5, atol=1e-12)
    # and the plain 2-norm is not the invariant for D3Q19: Gamma(1/2) is not unitary
    G = an.gamma_symbol(s, 0.5, [0.7, 0.2, -1.1])
    assert np.abs(G.conj().T @ G - np.eye(19)).max() > 1e-3


# --------------------------------------------------------------------------------------------
# the step
# --------------------------------------------------------------------------------------------

@pytest.mark.parametrize("name,shape", [("D1Q3", (5, 1, 1)), ("D2Q5", (4, 3, 1)), ("D2Q5_DI", (3, 4, 1)),
                                        ("D3Q7", (3, 3, 2)), ("D3Q7_DI", (2, 3, 3)), ("D3Q9", (3, 2, 2)),
                                        ("D3Q13", (2, 2, 3)), ("D3Q19", (3, 3, 3))])
def test_step_equals_assembled_step_matrix(name, shape):
    """Brute force on tiny periodic grids: n oracle steps equal M^n g with M = S (I (x) H(tau))
    assembled explicitly from the printed H and the periodic shift."""
    s = oracle.velset(name)
    cells = int(np.prod(shape))
    rng = np.random.default_rng(5)
    g = rng.normal(size=(s.q, cells))
    for tau in (0.5, 0.73):
        M = an.step_matrix(s, shape, tau)
        want = g.ravel()
        for n in (1, 2, 3):
            want = M @ want
            got = oracle.step(name, shape, tau, g, n)
            np.testing.assert_allclose(got.ravel(), want, atol=1e-13, rtol=0)


def test_d1q3_is_exact_dalembert_at_config_size():
    """The 1D configuration (N = 1024, tau = 0.8, Gaussian pulse of amplitude 1e-3 and width 20
    cells, 2000 steps) reproduces the closed-form d'Alembert solution to rounding (Sec. 9.1:
    errors close to machine precision)."""
    N, A, w = 1024, 1e-3, 20.0
    x = np.arange(N)
    x0 = 417.3
    dx = (x - x0 + N / 2) % N - N / 2
    G = A * np.exp(-(dx ** 2) / w ** 2)
    g = oracle.equilibrium("D1Q3", G, np.zeros((1, N)), np.zeros(N))
    g = oracle.step("D1Q3", (N, 1, 1), 0.8, g, 2000)
    rho, u, th = oracle.moments("D1Q3", g)
    want = an.dalembert_d1q3(G, 2000)
    # H = I only up to rounding: each step's moments/equilibrium round-trip adds O(1e-16) of the
    # amplitude, so after 2000 steps the error stays below 2000 * 2.5e-16 * A
    assert np.abs(rho - want).max() <= 5e-13 * A
    # velocity: the two acoustic halves carry u' = +-(c_s / rho0) rho'_acoustic
    wr = (0.5 / 3) * np.roll(G, 2000)
    wl = (0.5 / 3) * np.roll(G, -2000)
    assert np.abs(u[0] - (wr - wl)).max() <= 5e-13 * A


def test_d1q3_open_boundary_lets_the_pulse_leave():
    """D1Q3 with zero-incoming open edges: the same d'Alembert split, with the pulse continued by
    zero outside the grid, so the halves leave without reflection."""
    N = 200
    x = np.arange(N)
    G = np.exp(-((x - 80.0) ** 2) / 12.0 ** 2)
    g = oracle.equilibrium("D1Q3", G, np.zeros((1, N)), np.zeros(N))
    for t in (10, 150, 400):
        gt = oracle.step("D1Q3", (N, 1, 1), 0.8, g, t, bc="open_zero")
        rho = oracle.moments("D1Q3", gt)[0]
        ext = np.concatenate([np.zeros(t), G, np.zeros(t)])
        right = ext[t - t: t - t + N]  # G(x - t), zero outside
        left = ext[2 * t: 2 * t + N]   # G(x + t)
        np.testing.assert_allclose(rho, 2 / 3 * G + (right + left) / 6, atol=1e-15)


@pytest.mark.parametrize("name", ALL_SETS)
def test_exact_conservation_on_periodic_grids(name):
    """Collision keeps each cell's moments and streaming permutes populations, so total density,
    momentum and energy moment do not change (Secs. 4-6)."""
    s = oracle.velset(name)
    shape = grid_shape(s.D, (9, 7, 5))
    cells = int(np.prod(shape))
    rng = np.random.default_rng(8)
    g = rng.normal(size=(s.q, cells))
    r0 = oracle.reduce(name, g)
    g2 = oracle.step(name, shape, 0.62, g, 25)
    r1 = oracle.reduce(name, g2)
    scale = np.abs(g).sum()
    np.testing.assert_allclose(r1[: s.D + 2], r0[: s.D + 2], atol=1e-14 * scale)
    assert r1[-1] == 0


@pytest.mark.parametrize("name", ALL_SETS)
def test_weighted_energy_nonincreasing_iff_tau_ge_half(name):
    """H(tau) = (1 - 1/tau) I + (1/tau) P with P a projection that is self-adjoint for the weight
    diag(1/f*) (the A0 structure of Sec. 8.3.1), and streaming keeps that weighted norm: so
    E = sum g^2 / f* never grows for tau >= 1/2, is exactly conserved at tau = 1/2, and grows for
    tau < 1/2 (|1 - 1/tau| > 1)."""
    s = oracle.velset(name)
    shape = grid_shape(s.D, (8, 6, 4))
    cells = int(np.prod(shape))
    rng = np.random.default_rng(21)
    g = rng.normal(size=(s.q, cells))
    E0 = oracle.reduce(name, g)[s.D + 2]
    # tau = 1/2: conserved
    gh = oracle.step(name, shape, 0.5, g, 12)
    assert oracle.reduce(name, gh)[s.D + 2] == pytest.approx(E0, rel=1e-12)
    for tau in (0.52, 0.8, 1.5):
        prev = E0
        gt = g
        for _ in range(4):
            gt = oracle.step(name, shape, tau, gt, 2)
            E = oracle.reduce(name, gt)[s.D + 2]
            assert E <= prev * (1 + 1e-13)
            prev = E
    if s.q > s.D + 2:  # a non-conserved mode exists
        gb = oracle.step(name, shape, 0.45, g, 4)
        assert oracle.reduce(name, gb)[s.D + 2] > E0 * 1.01


@pytest.mark.parametrize("name", ["D1Q3", "D2Q5", "D2Q5_DI", "D3Q7", "D3Q19", "D3Q7_DI"])
def test_fourier_eigenmodes_evolve_by_their_eigenvalue(name):
    """Sec. 7: a population field Re(v e^{i k.x}) with v an eigenvector of Gamma(k) = D(k) H(tau)
    is, after n steps, Re(lambda^n v e^{i k.x}); and rho(Gamma) <= 1 (Theorem 1, condition 2)."""
    s = oracle.velset(name)
    shape = grid_shape(s.D, (8, 6, 4))
    nx, ny, nz = shape
    cells = nx * ny * nz
    X = np.stack(np.meshgrid(np.arange(nx), np.arange(ny), np.arange(nz), indexing="ij"), 0)
    X = X.transpose(0, 3, 2, 1).reshape(3, cells)  # cell = x + nx (y + ny z)
    for tau in (0.5, 0.7):
        m = np.array([1, 2, 1])
        k = 2 * np.pi * m / np.array(shape)
        k[s.D:] = 0.0
        lam, V = np.linalg.eig(an.gamma_symbol(s, tau, k[: s.D]))
        assert np.abs(lam).max() <= 1 + 1e-12
        phase = np.exp(1j * (k @ X))
        for j in range(s.q):
            v = V[:, j]
            g0 = np.real(v[:, None] * phase[None, :])
            n = 5
            got = oracle.step(name, shape, tau, g0, n)
            want = np.real(lam[j] ** n * v[:, None] * phase[None, :])
            np.testing.assert_allclose(got, want, atol=1e-13)


def test_spectral_reference_reproduces_a_plane_wave():
    """The exact-solution helper against the closed-form acoustic plane wave
    rho' = A cos(k.x - w t), u' = A c_s/rho0 k^ cos(.), theta' = (gamma-1) theta0 A / rho0 cos(.)."""
    s = oracle.velset("D2Q5_DI")
    nx, ny = 32, 16
    xs, ys = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    k = np.array([2 * np.pi * 3 / nx, 2 * np.pi * 2 / ny])
    kh = k / np.linalg.norm(k)
    cs = np.sqrt(s.cs2)
    A = 1e-3
    ph = lambda t: k[0] * xs + k[1] * ys - cs * np.linalg.norm(k) * t  # noqa: E731
    rho = A * np.cos(ph(0)).ravel()
    u = np.stack([A * cs / s.rho0 * kh[a] * np.cos(ph(0)).ravel() for a in range(2)])
    th = (s.gamma - 1) * s.theta0 * A / s.rho0 * np.cos(ph(0)).ravel()
    r, uu, tt = an.lee_spectral(s, (nx, ny, 1), rho, u, th, 7.3)
    np.testing.assert_allclose(r, A * np.cos(ph(7.3)).ravel(), atol=1e-15)
    np.testing.assert_allclose(uu[0], A * cs / s.rho0 * kh[0] * np.cos(ph(7.3)).ravel(), atol=1e-15)
    np.testing.assert_allclose(tt, (s.gamma - 1) * s.theta0 * A / s.rho0 * np.cos(ph(7.3)).ravel(), atol=1e-15)


def _convergence_errors(name, Ns, tau, L=2.0, T=0.5, a=20.0):
    """Gauss pulse rho' = exp(-a |x - centre|^2) on [0, L)^D (the IC form of Sec. 9), u' = theta' = 0,
    run to physical time T with epsilon = dx = dt = L/N; L2 error of rho' in the space norm of
    Sec. 9 against the exact LEE solution."""
    s = oracle.velset(name)
    errs = []
    for N in Ns:
        eps = L / N
        shape = grid_shape(s.D, (N, N, N))
        coords = np.meshgrid(*[np.arange(N) * eps for _ in range(s.D)], indexing="ij")
        r2 = sum((c - L / 2) ** 2 for c in coords)
        rho = np.exp(-a * r2)
        rho = rho.transpose(*reversed(range(s.D))).ravel()  # x fastest
        cells = rho.size
        u = np.zeros((s.D, cells))
        th = np.zeros(cells)
        g = oracle.equilibrium(name, rho, u, th)
        nsteps = int(round(T / eps))
        g = oracle.step(name, shape, tau, g, nsteps)
        r = oracle.moments(name, g)[0]
        ref = an.lee_spectral(s, shape, rho, u, th, nsteps)[0]
        errs.append(np.sqrt(np.sum((r - ref) ** 2) * eps ** s.D))
    return np.array(errs)


@pytest.mark.parametrize("name", ["D2Q5", "D2Q5_DI"])
def test_second_order_at_tau_half_first_order_otherwise(name):
    """Sec. 7: tau = 1/2 gives second-order consistency; for tau != 1/2 the (1/2 - tau) terms of
    the epsilon^2 moment equations survive and the scheme is first order."""
    Ns = [32, 64, 128]
    e = _convergence_errors(name, Ns, 0.5)
    order = np.log2(e[:-1] / e[1:])
    assert order[-1] > 1.8, (e, order)
    e1 = _convergence_errors(name, Ns, 0.6)
    order1 = np.log2(e1[:-1] / e1[1:])
    assert 0.8 < order1[-1] < 1.3, (e1, order1)


@pytest.mark.parametrize("name", ["D3Q7", "D3Q7_DI"])
def test_second_order_3d(name):
    e = _convergence_errors(name, [16, 32], 0.5, a=12.0)
    assert np.log2(e[0] / e[1]) > 1.7, e


# --------------------------------------------------------------------------------------------
# open boundaries
# --------------------------------------------------------------------------------------------

def test_ghost_boundary_reproduces_periodic_step():
    """Feeding the open-ghost edge with exactly the post-collision populations that a periodic grid
    would stream in reproduces the periodic step: pins edge and direction indexing of the ghost
    layout."""
    name = "D2Q5"
    nx, ny = 7, 5
    rng = np.random.default_rng(2)
    g = rng.normal(size=(5, nx * ny))
    tau = 0.7
    post = oracle.collide(name, tau, g).reshape(5, ny, nx)
    s = oracle.velset(name)
    L = max(nx, ny)
    ghost = np.zeros((4, L))
    idx = {tuple(c[:2]): i for i, c in enumerate(s.c)}
    ghost[0, :ny] = post[idx[(1, 0)], :, nx - 1]
    ghost[1, :ny] = post[idx[(-1, 0)], :, 0]
    ghost[2, :nx] = post[idx[(0, 1)], ny - 1, :]
    ghost[3, :nx] = post[idx[(0, -1)], 0, :]
    want = oracle.step(name, (nx, ny, 1), tau, g, 1)
    got = oracle.step(name, (nx, ny, 1), tau, g, 1, bc="open_ghost", ghost=ghost)
    np.testing.assert_allclose(got, want, atol=1e-15)


def test_sponge_profile_and_limits():
    """Sponge frame: zero strength equals the zero-incoming open edge; damping only touches frame
    cells; the weighted energy never grows for tau >= 1/2."""
    name = "D2Q5"
    nx, ny, w = 20, 16, 4
    rng = np.random.default_rng(4)
    g = rng.normal(size=(5, nx * ny))
    a = oracle.step(name, (nx, ny, 1), 0.6, g, 3, bc="open_zero")
    b = oracle.step(name, (nx, ny, 1), 0.6, g, 3, bc="open_sponge", sponge_w=w, sponge_smax=0.0)
    np.testing.assert_allclose(a, b, atol=0)
    # one step with a strong sponge: an equilibrium at rest in the interior is untouched there
    rho = np.zeros((ny, nx))
    rho[w + 2: ny - w - 2, w + 2: nx - w - 2] = 1.0
    ge = oracle.equilibrium(name, rho.ravel(), np.zeros((2, nx * ny)), np.zeros(nx * ny))
    e_prev = oracle.reduce(name, g)[4]
    gs = g
    for _ in range(5):
        gs = oracle.step(name, (nx, ny, 1), 0.55, gs, 1, bc="open_sponge", sponge_w=w, sponge_smax=0.5)
        e = oracle.reduce(name, gs)[4]
        assert e <= e_prev * (1 + 1e-13)
        e_prev = e
    one = oracle.step(name, (nx, ny, 1), 0.9, ge, 1, bc="open_sponge", sponge_w=w, sponge_smax=0.5)
    inner = (slice(None), slice(w + 3, ny - w - 3), slice(w + 3, nx - w - 3))
    np.testing.assert_allclose(one.reshape(5, ny, nx)[inner], ge.reshape(5, ny, nx)[inner], atol=1e-15)
    # outermost frame cell of a uniform field loses exactly sigma = smax of its post-collision value
    gu = oracle.equilibrium(name, np.ones(nx * ny), np.zeros((2, nx * ny)), np.zeros(nx * ny))
    one = oracle.step(name, (nx, ny, 1), 1.0, gu, 1, bc="open_sponge", sponge_w=w, sponge_smax=0.5)
    rest = one.reshape(5, ny, nx)[0]
    assert rest[0, 0] == pytest.approx(0.5 * 0.5, abs=1e-15)       # d = 4 = w -> sigma = 0.5
    assert rest[ny // 2, 1] == pytest.approx(0.5 * (1 - 0.5 * (3 / 4) ** 2), abs=1e-15)
    assert rest[ny // 2, w] == pytest.approx(0.5, abs=1e-15)       # first interior cell: no damping
